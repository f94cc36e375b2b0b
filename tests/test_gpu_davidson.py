"""Block Davidson on the GPU against the oracle: brute-force dense
diagonalisation for small cells, the oracle's own FP64 Davidson for larger ones;
residuals recomputed in FP64 by the oracle's H.  FP64 bar: eigenvalues within
1e-10 Ha of the oracle; mixed (reduced-precision phase, then FP64): 1e-8 Ha."""
import numpy as np
import pytest

from oracle import davidson as od
from oracle import hamiltonian as oh
from paper_1709_10010_gb300 import synthetic as syn
from tests.helpers import case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    from paper_1709_10010_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def system(cell, v, beta, D, precision="fp64"):
    import paper_1709_10010_gb300 as pwh
    s = pwh.System.from_cell(cell, precision=precision)
    s.set_potential(v)
    s.set_projectors(beta, D)
    return s


SMALL = [
    (dict(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1), 8),
    (dict(seed=2, a=9.0, natoms=3, ecut_ry=12.0, lmax=2, k=(0.25, -0.25, 0.25)), 10),
    (dict(seed=4, a=7.0, natoms=2, ecut_ry=10.0, lmax=1, k=(0.1, 0.3, -0.2)), 5),
]


@pytest.mark.parametrize("kw,nb", SMALL)
@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_jd"])
def test_davidson_matches_dense_eigh(torch, kw, nb, mode):
    cell, b, v, beta, D = case(**kw)
    H = oh.dense_h(b, v, beta, D)
    ex = np.linalg.eigvalsh(H)[:nb]
    s = system(cell, v, beta, D, precision="fp64" if mode == "fp64" else "mixed")
    psi0 = syn.initial_bands(3, b.npw, nb)
    psi = torch.from_numpy(psi0).cuda()
    tol = 1e-10 if mode == "fp64" else 1e-9
    eig, st, status = s.davidson(psi, tol=tol, mixed=(mode != "fp64"), switch_tol=1e-5,
                                 jd_inner=10 if mode == "mixed_jd" else 0)
    assert status == 0 and st["max_resid"] <= tol
    bar = 1e-10 if mode == "fp64" else 1e-8
    assert np.abs(eig - ex).max() <= bar, (eig - ex)
    X = psi.cpu().numpy()                      # (nb, npw) eigenvectors, public order
    assert np.abs(X.conj() @ X.T - np.eye(nb)).max() < 1e-10
    r = np.linalg.norm(H @ X.T - X.T * eig[None, :], axis=0)
    assert r.max() <= 2 * tol
    if mode != "fp64":
        assert st["switch_iter"] >= 1 and st["n_apply"] > st["n_apply_fp64"]


def test_davidson_small_workload_vs_oracle(torch):
    """The 1503-plane-wave cell (a=10, 20 Ry, 8 atoms, s+p projectors), lowest 16
    bands to 1e-8: GPU FP64 and mixed vs the dense oracle spectrum."""
    cfg = syn.CONFIGS["small"]
    cell, b, v, beta, D = case(seed=0, a=cfg["a"], natoms=cfg["natoms"], ecut_ry=cfg["ecut_ry"],
                               lmax=cfg["lmax"])
    assert b.npw == 1503
    nb = cfg["nb"]
    ex = np.linalg.eigvalsh(oh.dense_h(b, v, beta, D))[:nb]
    for mode in ("fp64", "mixed", "mixed_jd"):
        s = system(cell, v, beta, D, precision="fp64" if mode == "fp64" else "mixed")
        psi = torch.from_numpy(syn.initial_bands(0, b.npw, nb)).cuda()
        eig, st, status = s.davidson(psi, tol=1e-8, mixed=(mode != "fp64"),
                                     jd_inner=10 if mode == "mixed_jd" else 0)
        assert status == 0
        assert np.abs(eig - ex).max() <= 1e-8
        # residual recomputed by the oracle's FP64 operator
        X = psi.cpu().numpy()
        r = np.linalg.norm(oh.apply_h(b, v, beta, D, X) - X * eig[:, None], axis=1)
        assert r.max() <= 2e-8


def test_davidson_no_preconditioner_and_tight_subspace(torch):
    cell, b, v, beta, D = case(seed=5, a=8.0, natoms=3, ecut_ry=12.0, lmax=1)
    nb = 6
    ex = np.linalg.eigvalsh(oh.dense_h(b, v, beta, D))[:nb]
    s = system(cell, v, beta, D)
    for precond, mult in (("none", 2), ("tpa", 2), ("tpa", 5)):
        psi = torch.from_numpy(syn.initial_bands(7, b.npw, nb)).cuda()
        eig, st, status = s.davidson(psi, tol=1e-9, precond=precond, mult=mult, max_iter=500)
        assert status == 0
        assert np.abs(eig - ex).max() <= 1e-9


def test_davidson_free_electrons_degenerate(torch):
    """V = 0, no projectors: the spectrum is the sorted kinetic energies with the
    degenerate shells 1, 6, 12, ... (band cut inside the 12-fold shell)."""
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(seed=6, a=7.0, natoms=1, ecut_ry=10.0, lmax=0)
    s = pwh.System.from_cell(cell)
    s.set_potential(np.zeros(b.fft))
    nb = 12
    psi = torch.from_numpy(syn.initial_bands(8, b.npw, nb)).cuda()
    eig, st, status = s.davidson(psi, tol=1e-10)
    assert status == 0
    np.testing.assert_allclose(eig, np.sort(b.kinetic)[:nb], atol=1e-10)


def test_davidson_not_converged_status(torch):
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(seed=0)
    s = system(cell, v, beta, D)
    psi = torch.from_numpy(syn.initial_bands(1, b.npw, 4)).cuda()
    eig, st, status = s.davidson(psi, tol=1e-12, max_iter=1, check=False)
    assert status == 4 and st["iters"] == 1
    assert np.all(np.isfinite(eig))
    # invalid options are host-side argument errors
    with pytest.raises(pwh.PwhError) as e:
        s.davidson(psi, tol=-1.0)
    assert e.value.status == 1


def test_davidson_medium_vs_oracle_davidson(torch):
    """The 34,265-plane-wave cell, lowest 32 bands: GPU FP64 vs the oracle's own
    FP64 Davidson (no dense route at this size); agreement of the two
    independent solvers within 1e-8 Ha, residual bound of the GPU result
    recomputed by the oracle."""
    cell = syn.config_cell("medium", 0)
    from oracle import basis as ob
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    nb = 32
    X0 = syn.initial_bands(0, b.npw, nb)
    s = system(cell, v, beta, D)
    psi = torch.from_numpy(X0).cuda()
    eig, st, status = s.davidson(psi, tol=1e-8)
    assert status == 0
    res = od.davidson(lambda X: oh.apply_h(b, v, beta, D, X.T).T, b.kinetic, X0.T, nb, tol=1e-8,
                      m_max=3 * nb)
    assert res.converged
    assert np.abs(eig - res.eig).max() <= 1e-8
    X = psi.cpu().numpy()
    r = np.linalg.norm(oh.apply_h(b, v, beta, D, X) - X * eig[:, None], axis=1)
    assert r.max() <= 2e-8
