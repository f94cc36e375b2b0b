"""Pins of the oracle's H|psi> (CPU only): closed forms, brute force, library
routines and invariants of the plane-wave Hamiltonian."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

from oracle import basis as ob
from oracle import hamiltonian as oh
from paper_1709_10010_gb300 import synthetic as syn


def tiny(seed=0, a=6.0, natoms=2, ecut_ry=8.0, lmax=1, k=(0, 0, 0)):
    cell = syn.make_cell(seed, a, natoms, ecut_ry, lmax, kpoint=k)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    return cell, b, v, beta, D


def test_vtilde_is_naive_dft():
    rng = np.random.default_rng(3)
    n = (4, 5, 6)
    v = rng.standard_normal(n)
    vt = oh.v_tilde(v)
    j = np.stack(np.meshgrid(*[np.arange(x) for x in n], indexing="ij"), -1).reshape(-1, 3)
    for m in [(0, 0, 0), (1, 2, 3), (3, 4, 5), (2, 0, 1)]:
        ph = np.exp(-2j * np.pi * (j[:, 0] * m[0] / n[0] + j[:, 1] * m[1] / n[1] + j[:, 2] * m[2] / n[2]))
        ref = (v.reshape(-1) * ph).sum() / v.size
        assert abs(vt[m] - ref) < 1e-14


def test_free_electrons_closed_form():
    """V = 0, no projectors: H psi = 1/2|k+G|^2 psi and the eigenvalues are the
    sorted 1/2|k+G|^2."""
    cell, b, v, beta, D = tiny(k=(0.1, -0.2, 0.3))
    psi = syn.initial_bands(1, b.npw, 3)
    hp = oh.apply_h(b, np.zeros(b.fft), None, None, psi)
    np.testing.assert_allclose(hp, b.kinetic[None] * psi, rtol=0, atol=1e-14)
    ev = np.linalg.eigvalsh(oh.dense_h(b, np.zeros(b.fft), None, None))
    np.testing.assert_allclose(ev, np.sort(b.kinetic), rtol=0, atol=1e-13)


def test_constant_potential_shifts_spectrum():
    cell, b, v, beta, D = tiny()
    c = -0.731
    psi = syn.initial_bands(2, b.npw, 2)
    h0 = oh.apply_h(b, v, beta, D, psi)
    h1 = oh.apply_h(b, v + c, beta, D, psi)
    np.testing.assert_allclose(h1 - h0, c * psi, rtol=0, atol=1e-12)
    e0 = np.linalg.eigvalsh(oh.dense_h(b, v, beta, D))
    e1 = np.linalg.eigvalsh(oh.dense_h(b, v + c, beta, D))
    np.testing.assert_allclose(e1 - e0, c, rtol=0, atol=1e-11)


def test_cosine_potential_closed_form():
    """V(r) = cos(g0.r) couples G to G +- g0 with weight 1/2 (checks FFT signs,
    scaling and index wrap of the local route)."""
    cell, b, v, beta, D = tiny(a=5.0, ecut_ry=10.0)
    n = b.fft
    g0 = (1, 2, 0)
    i = np.stack(np.meshgrid(*[np.arange(x) for x in n], indexing="ij"), -1)
    vr = np.cos(2 * np.pi * (i[..., 0] * g0[0] / n[0] + i[..., 1] * g0[1] / n[1] + i[..., 2] * g0[2] / n[2]))
    psi = syn.initial_bands(4, b.npw, 2)
    where = {tuple(m): j for j, m in enumerate(b.miller)}
    ref = np.zeros_like(psi)
    for j, m in enumerate(b.miller):
        for s in (+1, -1):
            src = (m[0] - s * g0[0], m[1] - s * g0[1], m[2] - s * g0[2])
            if src in where:
                ref[:, j] += 0.5 * psi[:, where[src]]
    for route in (oh.local_fft, oh.local_dense):
        np.testing.assert_allclose(route(b.miller, n, vr, psi), ref, rtol=0, atol=1e-13)
    # sin(g0.r) = (e^{+i g0.r} - e^{-i g0.r}) / 2i is odd: it pins the FFT sign
    vs = np.sin(2 * np.pi * (i[..., 0] * g0[0] / n[0] + i[..., 1] * g0[1] / n[1] + i[..., 2] * g0[2] / n[2]))
    ref = np.zeros_like(psi)
    for j, m in enumerate(b.miller):
        for s in (+1, -1):
            src = (m[0] - s * g0[0], m[1] - s * g0[1], m[2] - s * g0[2])
            if src in where:
                ref[:, j] += s * psi[:, where[src]] / 2j
    for route in (oh.local_fft, oh.local_dense):
        np.testing.assert_allclose(route(b.miller, n, vs, psi), ref, rtol=0, atol=1e-13)


def test_parseval_and_unit_potential():
    """V = 1 is the identity on the sphere; the inverse FFT obeys
    sum_r |psi(r)|^2 = N^3 sum_G |c_G|^2."""
    cell, b, v, beta, D = tiny()
    psi = syn.initial_bands(5, b.npw, 2)
    np.testing.assert_allclose(oh.local_fft(b.miller, b.fft, np.ones(b.fft), psi), psi, atol=1e-13)
    n1, n2, n3 = b.fft
    box = np.zeros(b.fft, dtype=complex)
    box[b.miller[:, 0] % n1, b.miller[:, 1] % n2, b.miller[:, 2] % n3] = psi[0]
    pr = np.fft.ifftn(box) * box.size
    assert abs((np.abs(pr) ** 2).sum() - box.size * (np.abs(psi[0]) ** 2).sum()) < 1e-9 * box.size


@pytest.mark.parametrize("k", [(0, 0, 0), (0.25, -0.25, 0.25)])
def test_dense_and_fft_routes_agree(k):
    cell, b, v, beta, D = tiny(seed=7, a=8.0, natoms=3, ecut_ry=12.0, lmax=2, k=k)
    psi = syn.initial_bands(6, b.npw, 3)
    hf = oh.apply_h(b, v, beta, D, psi, route="fft")
    hd = oh.apply_h(b, v, beta, D, psi, route="dense")
    assert np.abs(hf - hd).max() <= 1e-13 * np.abs(hd).max()
    hm = (oh.dense_h(b, v, beta, D) @ psi.T).T
    assert np.abs(hm - hd).max() <= 1e-13 * np.abs(hd).max()


def test_hermiticity():
    cell, b, v, beta, D = tiny(seed=8, lmax=2, k=(0.25, 0.25, -0.25))
    x = syn.initial_bands(9, b.npw, 2)
    hx = oh.apply_h(b, v, beta, D, x)
    lhs = np.vdot(x[0], hx[1])
    rhs = np.conj(np.vdot(x[1], hx[0]))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_single_projector_secular_equation():
    """V = 0, one s projector with coefficient d: every eigenvalue eps not equal to a
    kinetic level solves 1 = d sum_G |beta_G|^2 / (eps - T_G) (rank-one update)."""
    cell = syn.make_cell(11, 6.0, 1, 10.0, 0)
    cell.d_l[:] = 0.8
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    ev = np.linalg.eigvalsh(oh.dense_h(b, np.zeros(b.fft), beta, D))
    w = np.abs(beta[0]) ** 2
    levels = np.unique(np.round(b.kinetic, 12))

    def f(e):
        return 1.0 - 0.8 * np.sum(w / (e - b.kinetic))
    # bisection for the root above the lowest level (d > 0 pushes it up)
    lo, hi = levels[0] + 1e-12, levels[1] - 1e-12
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(lo) * f(mid) <= 0:
            hi = mid
        else:
            lo = mid
    root = 0.5 * (lo + hi)
    assert np.min(np.abs(ev - root)) < 1e-10


def test_projector_radial_transform_by_quadrature():
    """The analytic Gaussian transform against numerical quadrature of
    4 pi int r^2 j_l(qr) r^l exp(-r^2/2) dr (rc = 1)."""
    for l in (0, 1, 2):
        for q in (0.3, 1.1, 2.7):
            num = scipy.integrate.quad(lambda r: r ** 2 * scipy.special.spherical_jn(l, q * r)
                                       * r ** l * math.exp(-0.5 * r * r), 0, 40, limit=200)[0]
            ana = math.sqrt(math.pi / 2) * q ** l * math.exp(-0.5 * q * q)
            assert abs(num - ana) < 1e-10


def _eigs(cell, nb, fft=None):
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha, fft=fft)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    return np.linalg.eigvalsh(oh.dense_h(b, v, beta, syn.d_diagonal(cell)))[:nb]


def test_invariant_translation():
    cell = syn.make_cell(12, 6.0, 2, 10.0, 2)
    e0 = _eigs(cell, 8)
    cell.positions = cell.positions + np.array([0.37, -1.2, 2.05])
    e1 = _eigs(cell, 8)
    np.testing.assert_allclose(e0, e1, atol=1e-9)


def test_invariant_time_reversal():
    cell = syn.make_cell(13, 6.0, 2, 10.0, 2, kpoint=(0.25, -0.25, 0.25))
    e0 = _eigs(cell, 8)
    cell.kpoint = -cell.kpoint
    np.testing.assert_allclose(e0, _eigs(cell, 8), atol=1e-11)


def test_invariant_nested_basis_interlacing():
    cell = syn.make_cell(14, 6.0, 2, 8.0, 1)
    e_lo = _eigs(cell, 8, fft=(24, 24, 24))
    cell.ecut_ha = 6.0
    e_hi = _eigs(cell, 8, fft=(24, 24, 24))
    assert np.all(e_hi <= e_lo + 1e-12)
    assert np.any(e_hi < e_lo - 1e-8)


def test_invariant_cubic_rotation():
    """Rotating every atom by 90 degrees about z (a cubic point-group operation)
    with D shared over m leaves the spectrum unchanged."""
    cell = syn.make_cell(15, 6.0, 2, 10.0, 2)
    e0 = _eigs(cell, 8)
    p = cell.positions.copy()
    cell.positions = np.stack([-p[:, 1], p[:, 0], p[:, 2]], axis=1) % 6.0
    np.testing.assert_allclose(e0, _eigs(cell, 8), atol=1e-9)
