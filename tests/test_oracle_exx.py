"""Pins of the oracle's exact exchange and ACE (CPU only).

* The FFT route against the reciprocal-space sum with no FFT (cubic and
  skewed cells, k = 0 and a shifted k).
* Closed form: one occupied plane wave e_G1 acting on e_G2 gives
  -4 pi f / (Omega |G2 - G1|^2) e_G2, and nothing for G2 = G1.
* V_x is Hermitian and negative semidefinite, linear in the weights, and
  invariant under a unitary mixing of equally weighted occupied bands (a
  missing conjugate in the pair density breaks this).
* ACE equals V_x on the occupied bands, equals xi M^-1 xi^H of Eq. Vxace (by a
  linear solve, no Cholesky) on any band, and is negative semidefinite of rank
  nocc.
"""
import numpy as np
import pytest

from oracle import basis as ob
from oracle import exx
from paper_1709_10010_gb300 import synthetic as syn


def small_case(skew=False, k=(0.0, 0.0, 0.0)):
    lat = np.array([[6.0, 0.0, 0.0], [0.7, 5.5, 0.0], [0.3, -0.4, 6.2]]) if skew else 6.0
    cell = syn.make_cell(0, lat, 2, 6.0, 1, kpoint=k)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    return cell, b


def orthonormal_bands(seed, npw, n):
    q, _ = np.linalg.qr(syn.initial_bands(seed, npw, n).T)
    return q.T


@pytest.mark.parametrize("skew,k", [(False, (0, 0, 0)), (True, (0, 0, 0)), (True, (0.25, -0.1, 0.3))])
def test_fft_route_matches_reciprocal_sum(skew, k):
    cell, b = small_case(skew, k)
    psi = orthonormal_bands(1, b.npw, 3)
    phi = syn.initial_bands(2, b.npw, 2)
    occ = np.array([2.0, 1.0, 0.5])
    a = exx.exchange(b, cell.lattice, psi, occ, phi)
    c = exx.exchange_brute(b, cell.lattice, psi, occ, phi)
    assert np.abs(a - c).max() <= 1e-13 * np.abs(c).max()


def test_single_plane_wave_closed_form():
    cell, b = small_case(True, (0.1, 0.0, -0.2))
    volume = abs(np.linalg.det(cell.lattice))
    bvec = ob.reciprocal(cell.lattice)
    i1, i2 = 3, 11
    psi = np.zeros((1, b.npw), complex)
    psi[0, i1] = 1.0
    phi = np.zeros((1, b.npw), complex)
    phi[0, i2] = 0.7 - 0.2j
    out = exx.exchange(b, cell.lattice, psi, np.array([1.5]), phi)
    q = (b.miller[i2] - b.miller[i1]) @ bvec
    ref = -4.0 * np.pi * 1.5 / (volume * float(q @ q)) * phi
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-14 * np.abs(ref).max())
    same = exx.exchange(b, cell.lattice, psi, np.array([1.5]), psi)
    assert np.abs(same).max() <= 1e-15


def test_hermitian_negative_linear_and_unitary_invariant():
    cell, b = small_case(True, (0.25, 0.0, 0.0))
    psi = orthonormal_bands(3, b.npw, 4)
    occ = np.array([1.0, 1.0, 1.0, 1.0])
    A = syn.initial_bands(4, b.npw, 5)
    VA = exx.exchange(b, cell.lattice, psi, occ, A)
    G = np.conj(A) @ VA.T                        # G[m, n] = <a_m | V_x a_n>
    assert np.abs(G - G.conj().T).max() <= 1e-13 * np.abs(G).max()
    assert np.linalg.eigvalsh(0.5 * (G + G.conj().T)).max() <= 1e-13 * np.abs(G).max()
    # linear in the weights
    V2 = exx.exchange(b, cell.lattice, psi, 2.0 * occ, A)
    np.testing.assert_allclose(V2, 2.0 * VA, rtol=0, atol=1e-13 * np.abs(VA).max())
    # a unitary mixing of equally weighted occupied bands leaves V_x unchanged
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    VU = exx.exchange(b, cell.lattice, U.T @ psi, occ, A)
    np.testing.assert_allclose(VU, VA, rtol=0, atol=1e-13 * np.abs(VA).max())


def test_ace_exact_on_occupied_and_equal_to_eq_vxace():
    cell, b = small_case(False, (0, 0, 0))
    psi = orthonormal_bands(6, b.npw, 4)
    occ = np.array([2.0, 2.0, 1.0, 0.5])
    zeta = exx.ace(b, cell.lattice, psi, occ)
    assert zeta.shape == (4, b.npw)
    vx = exx.exchange(b, cell.lattice, psi, occ, psi)
    np.testing.assert_allclose(exx.apply_ace(zeta, psi), vx, rtol=0, atol=1e-12 * np.abs(vx).max())
    # Eq. Vxace written out: xi M^-1 xi^H phi with M = <psi_j | xi_m>, by a linear solve
    phi = syn.initial_bands(7, b.npw, 3)
    M = np.conj(psi) @ vx.T
    coef = np.linalg.solve(M, np.conj(vx) @ phi.T)          # M^-1 xi^H phi
    ref = (vx.T @ coef).T
    np.testing.assert_allclose(exx.apply_ace(zeta, phi), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # negative semidefinite, rank nocc, alpha scales it
    A = syn.initial_bands(8, b.npw, 8)
    G = np.conj(A) @ exx.apply_ace(zeta, A).T
    ev = np.linalg.eigvalsh(0.5 * (G + G.conj().T))
    assert ev.max() <= 1e-12 * np.abs(ev).max()
    assert np.sum(np.abs(ev) > 1e-10 * np.abs(ev).max()) == 4
    z4 = exx.ace(b, cell.lattice, psi, occ, alpha=0.25)
    np.testing.assert_allclose(exx.apply_ace(z4, phi), 0.25 * ref, rtol=0, atol=1e-12 * np.abs(ref).max())
