"""The overlap operator S = 1 + sum |beta_i> q_ij <beta_j| and the generalised
eigenproblem H x = e S x on the GPU against the oracle (oracle/overlap.py),
through the C ABI.  S psi: within 1e-12 of max |S psi|.  Eigenvalues against
LAPACK's generalised solver on the dense matrices: 1e-10 Ha (FP64), 1e-8 Ha
(mixed + Jacobi-Davidson); eigenvectors S-orthonormal, residual H x - e S x by
the oracle's operators."""
import numpy as np
import pytest

from oracle import basis as ob
from oracle import hamiltonian as oh
from oracle import overlap as oo
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


def q_of(P, seed, full):
    """Diagonal q_i ~ U(0.1, 0.8), or a full positive definite q (so S > 0)."""
    rng = np.random.default_rng(seed)
    if not full:
        return rng.uniform(0.1, 0.8, P)
    a = rng.standard_normal((P, P)) + 1j * rng.standard_normal((P, P))
    return 0.5 * (a @ a.conj().T) / P + 0.1 * np.eye(P)


CASES = [
    dict(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1),
    dict(seed=2, a=9.0, natoms=3, ecut_ry=12.0, lmax=2, k=(0.25, -0.25, 0.25)),
]


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("full", [False, True])
def test_apply_s_matches_oracle(torch, kw, full):
    cell, b, v, beta, D = case(**kw)
    s = make_system(cell, v, beta, D)
    q = q_of(beta.shape[0], 1, full)
    s.set_overlap(q)
    psi = syn.initial_bands(3, b.npw, 6)
    out = s.apply_s(torch.from_numpy(psi).cuda()).cpu().numpy()
    assert rel_err(out, oo.apply_s(beta, q, psi)) <= 1e-12
    # no overlap: the identity
    s.set_overlap(None)
    out0 = s.apply_s(torch.from_numpy(psi).cuda()).cpu().numpy()
    assert np.abs(out0 - psi).max() == 0.0


@pytest.mark.parametrize("kw,nb", [(CASES[0], 8), (CASES[1], 10)])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("full", [False, True])
def test_generalised_davidson_matches_lapack(torch, kw, nb, mode, full):
    cell, b, v, beta, D = case(**kw)
    s = make_system(cell, v, beta, D, mode)
    q = q_of(beta.shape[0], 4, full)
    s.set_overlap(q)
    H = oh.dense_h(b, v, beta, D)
    S = oo.dense_s(beta, q, b.npw)
    ref, _ = oo.gen_eigh(H, S, nb)
    psi = torch.from_numpy(syn.initial_bands(5, b.npw, nb)).cuda()
    mixed = mode == "mixed"
    eig, st, status = s.davidson(psi, tol=1e-9, mixed=mixed, switch_tol=1e-3,
                                 jd_inner=20 if mixed else 0)
    assert status == 0
    assert np.abs(eig - ref).max() <= (1e-10 if mode == "fp64" else 1e-8), np.abs(eig - ref).max()
    X = psi.cpu().numpy()
    assert np.abs(X.conj() @ S @ X.T - np.eye(nb)).max() < 1e-10
    R = oh.apply_h(b, v, beta, D, X) - eig[:, None] * oo.apply_s(beta, q, X)
    assert np.linalg.norm(R, axis=1).max() <= 1e-8


def test_zero_q_is_the_standard_problem(torch):
    cell, b, v, beta, D = case(**CASES[0])
    s = make_system(cell, v, beta, D)
    s.set_overlap(np.zeros(beta.shape[0]))
    psi = torch.from_numpy(syn.initial_bands(6, b.npw, 6)).cuda()
    eig, _, status = s.davidson(psi, tol=1e-10)
    assert status == 0
    ref = np.linalg.eigvalsh(oh.dense_h(b, v, beta, D))[:6]
    assert np.abs(eig - ref).max() <= 1e-10


def test_overlap_errors_and_resets(torch):
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(**CASES[0])
    s0 = pwh.System.from_cell(cell)
    s0.set_potential(v)
    with pytest.raises(pwh.PwhError) as e:          # no projectors yet
        s0.set_overlap(np.ones(beta.shape[0]))
    assert e.value.status == 7
    s = make_system(cell, v, beta, D)
    with pytest.raises(pwh.PwhError) as e:          # S not positive definite
        s.set_overlap(np.full(beta.shape[0], -50.0))
    assert e.value.status == 1
    psi = syn.initial_bands(7, b.npw, 3)
    assert np.abs(s.apply_s(torch.from_numpy(psi).cuda()).cpu().numpy() - psi).max() == 0.0
    s.set_overlap(np.full(beta.shape[0], 0.5))
    half = (b.npw + 1) // 2
    with pytest.raises(pwh.PwhError) as e:          # the real-band solver takes no overlap
        s.davidson_gamma(torch.zeros((3, half), dtype=torch.complex128, device="cuda"))
    assert e.value.status == 1
    s.set_projectors(beta, D)                       # new projectors drop the overlap
    assert np.abs(s.apply_s(torch.from_numpy(psi).cuda()).cpu().numpy() - psi).max() == 0.0


def test_generalised_medium_cell(torch):
    """The 34,265-plane-wave cell, 64 bands, mixed + Jacobi-Davidson with
    q_i ~ U(0.1, 0.8): S-orthonormal eigenvectors and residuals H x - e S x by
    the oracle's operators on sampled bands."""
    cell = syn.config_cell("medium", 0)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    s = make_system(cell, v, beta, D, "mixed")
    q = q_of(beta.shape[0], 8, False)
    s.set_overlap(q)
    nb = 64
    psi = torch.from_numpy(syn.initial_bands(0, b.npw, nb)).cuda()
    eig, st, status = s.davidson(psi, tol=1e-8, mixed=True, switch_tol=1e-3, jd_inner=20)
    assert status == 0
    X = psi.cpu().numpy()
    pick = [0, 1, 31, 62, 63]
    SX = oo.apply_s(beta, q, X[pick])
    assert np.abs(X[pick].conj() @ SX.T - np.eye(len(pick))).max() < 1e-10
    R = oh.apply_h(b, v, beta, D, X[pick]) - eig[pick, None] * SX
    assert np.linalg.norm(R, axis=1).max() <= 1e-7
    s.close()
