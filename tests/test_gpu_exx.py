"""Exact exchange and ACE on the GPU against the oracle (oracle/exx.py), through
the C ABI.  V_x: element by element within 1e-12 of max |V_x phi| (FP64 box
FFTs).  ACE inside H: the FP64 and mixed bars of the H|psi> tests (1e-12,
1e-4 of max |H psi|); eigenvalues of H + V_ACE against LAPACK on the dense
matrix (1e-10 FP64, 1e-8 mixed)."""
import numpy as np
import pytest

from oracle import basis as ob
from oracle import exx
from oracle import gamma as og
from oracle import hamiltonian as oh
from paper_1709_10010_gb300 import synthetic as syn
from tests.helpers import case, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    from paper_1709_10010_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def make_system(cell, v, beta, D, precision="fp64"):
    import paper_1709_10010_gb300 as pwh
    s = pwh.System.from_cell(cell, precision=precision)
    s.set_potential(v)
    s.set_projectors(beta, D)
    return s


def occupied(seed, npw, n):
    q, _ = np.linalg.qr(syn.initial_bands(seed, npw, n).T)
    return np.ascontiguousarray(q.T)


CASES = [
    dict(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1),
    dict(seed=2, a=9.0, natoms=3, ecut_ry=12.0, lmax=2, k=(0.25, -0.25, 0.25)),
    dict(seed=1, a=10.0, natoms=8, ecut_ry=20.0, lmax=1),     # the 1503-plane-wave cell
]


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("nocc,nb", [(1, 1), (4, 3), (9, 5)])
def test_exx_apply_matches_oracle(torch, kw, nocc, nb):
    cell, b, v, beta, D = case(**kw)
    s = make_system(cell, v, beta, D)
    psi = occupied(3 + nocc, b.npw, nocc)
    occ = np.linspace(2.0, 0.5, nocc)
    phi = syn.initial_bands(40 + nb, b.npw, nb)
    ref = exx.exchange(b, cell.lattice, psi, occ, phi)
    out = s.exx_apply(torch.from_numpy(psi).cuda(), occ, torch.from_numpy(phi).cuda()).cpu().numpy()
    assert rel_err(out, ref) <= 1e-12, rel_err(out, ref)


def test_exx_apply_skewed_cell(torch):
    lat = np.array([[8.0, 0.0, 0.0], [1.1, 7.4, 0.0], [0.6, -0.9, 8.3]])
    cell = syn.make_cell(7, lat, 3, 12.0, 1, kpoint=(0.1, 0.2, -0.3))
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    s = make_system(cell, syn.potential_grid(cell, b.fft), syn.projectors(cell, b.miller),
                    syn.d_diagonal(cell))
    psi = occupied(1, b.npw, 5)
    occ = np.full(5, 2.0)
    phi = syn.initial_bands(2, b.npw, 4)
    ref = exx.exchange(b, cell.lattice, psi, occ, phi)
    out = s.exx_apply(torch.from_numpy(psi).cuda(), occ, torch.from_numpy(phi).cuda()).cpu().numpy()
    assert rel_err(out, ref) <= 1e-12


@pytest.mark.parametrize("kw", CASES[:2])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_ace_inside_h(torch, kw, mode):
    """H with ACE against the oracle's H plus -zeta zeta^H; on the occupied
    bands the added term equals alpha V_x."""
    cell, b, v, beta, D = case(**kw)
    s = make_system(cell, v, beta, D, mode)
    nocc, alpha = 6, 0.25
    psi = occupied(11, b.npw, nocc)
    occ = np.full(nocc, 2.0)
    rank = s.set_ace(torch.from_numpy(psi).cuda(), occ, alpha)
    assert rank == nocc
    zeta = exx.ace(b, cell.lattice, psi, occ, alpha)
    phi = syn.initial_bands(12, b.npw, 7)
    ref = oh.apply_h(b, v, beta, D, phi) + exx.apply_ace(zeta, phi)
    out = s.apply_h(torch.from_numpy(phi).cuda()).cpu().numpy()
    s.sync()
    assert rel_err(out, ref) <= (1e-12 if mode == "fp64" else 1e-4), rel_err(out, ref)
    if mode == "fp64":
        h_occ = s.apply_h(torch.from_numpy(psi).cuda()).cpu().numpy()
        vx = exx.exchange(b, cell.lattice, psi, occ, psi)
        d = h_occ - oh.apply_h(b, v, beta, D, psi)
        assert rel_err(d, alpha * vx) <= 1e-11
    # removing the term restores H
    assert s.set_ace(None) == 0
    out0 = s.apply_h(torch.from_numpy(phi).cuda()).cpu().numpy()
    ref0 = oh.apply_h(b, v, beta, D, phi)
    assert rel_err(out0, ref0) <= (1e-12 if mode == "fp64" else 1e-4)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_davidson_with_ace_matches_dense_eigh(torch, mode):
    """Lowest eigenpairs of H + V_ACE (the inner loop of a hybrid-functional
    SCF) against LAPACK on the dense matrix."""
    cell, b, v, beta, D = case(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1)
    s = make_system(cell, v, beta, D, mode)
    H = oh.dense_h(b, v, beta, D)
    w, U = np.linalg.eigh(H)
    nocc = 4
    psi = np.ascontiguousarray(U[:, :nocc].T)            # occupied: lowest bands of H
    occ = np.full(nocc, 2.0)
    s.set_ace(torch.from_numpy(psi).cuda(), occ, 0.25)
    zeta = exx.ace(b, cell.lattice, psi, occ, 0.25)
    Hx = H - zeta.T @ np.conj(zeta)
    ref = np.linalg.eigvalsh(0.5 * (Hx + Hx.conj().T))[:8]
    start = torch.from_numpy(syn.initial_bands(5, b.npw, 8)).cuda()
    mixed = mode == "mixed"
    eig, st, status = s.davidson(start, tol=1e-9, mixed=mixed, switch_tol=1e-3,
                                 jd_inner=20 if mixed else 0)
    assert status == 0
    assert np.abs(eig - ref).max() <= (1e-10 if mode == "fp64" else 1e-8), np.abs(eig - ref).max()
    # exchange lowers the occupied levels: the lowest eigenvalue moves down
    assert eig[0] < w[0]


def test_ace_with_real_bands_at_gamma(torch):
    """Real occupied bands at k = 0 give real ACE projectors: the real-band
    route carries the term; complex occupied bands are refused there."""
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(seed=1, a=10.0, natoms=8, ecut_ry=20.0, lmax=1)
    s = make_system(cell, v, beta, D)
    half, _ = og.half_sphere(b.miller)
    nocc = 5
    h = syn.initial_bands(13, len(half), nocc)
    g0 = int(np.nonzero(np.all(b.miller[half] == 0, axis=1))[0][0])
    h[:, g0] = h[:, g0].real
    # real functions (ACE needs linearly independent bands, not orthonormal ones)
    q = og.expand(b.miller, h)
    q /= np.linalg.norm(q, axis=1)[:, None]
    occ = np.full(nocc, 2.0)
    s.set_ace(torch.from_numpy(q).cuda(), occ, 1.0)
    zeta = exx.ace(b, cell.lattice, q, occ, 1.0)
    phi = syn.initial_bands(14, len(half), 4)
    phi[:, g0] = phi[:, g0].real
    ref = (oh.apply_h(b, v, beta, D, og.expand(b.miller, phi)) +
           exx.apply_ace(zeta, og.expand(b.miller, phi)))[:, half]
    out = s.apply_h_gamma(torch.from_numpy(phi).cuda()).cpu().numpy()
    assert rel_err(out, ref) <= 1e-12
    # complex occupied bands: not real functions
    s.set_ace(torch.from_numpy(occupied(15, b.npw, 3)).cuda(), np.full(3, 2.0), 1.0)
    with pytest.raises(pwh.PwhError) as e:
        s.apply_h_gamma(torch.from_numpy(phi).cuda())
    assert e.value.status == 1


def test_ace_argument_errors(torch):
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1)
    s = make_system(cell, v, beta, D)
    psi = torch.from_numpy(occupied(1, b.npw, 3)).cuda()
    for occ, alpha in ((np.full(3, 2.0), 0.0), (np.array([2.0, -1.0, 2.0]), 1.0),
                       (np.array([2.0, np.nan, 2.0]), 1.0)):
        with pytest.raises(pwh.PwhError) as e:
            s.set_ace(psi, occ, alpha)
        assert e.value.status == 1
