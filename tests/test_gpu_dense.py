"""Subspace diagonalisation (device Jacobi, FP32 sweeps + FP64 polish) against
LAPACK (numpy.linalg.eigh): random, structured, degenerate and diagonal
matrices, odd and even sizes, on every FP32 stage (the 16-CTA cluster kernel
or the position-order kernel for 64 <= n <= 512, the block Jacobi over the
whole GPU beyond, the small cluster kernel below 64).  Bar: eigenvalues
within 1e-12 of max |lambda|, eigenvectors orthonormal and with residual
<= 1e-11 max |lambda|.  The FP32 result (precision="mixed"): eigenvalues within
2e-6 max |lambda|, orthonormality 2e-6, residual 2e-5 max |lambda| (about 30
FP32 roundings of the largest eigenvalue)."""
import numpy as np
import pytest

from paper_1709_10010_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1709_10010_gb300 as pwh
    from paper_1709_10010_gb300 import build
    build.build()
    s = pwh.System(np.diag([6.0] * 3), ecut_ha=2.0)
    return torch, s


def degenerate(n, seed):
    rng = np.random.default_rng(seed)
    levels = np.repeat([0.0, 0.4, 0.8, 1.2, 5.0], int(np.ceil(n / 5)))[:n]
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return (q * levels) @ q.conj().T


CASES = [("random", 12), ("random", 7), ("random", 96), ("random", 257), ("degenerate", 12),
         ("degenerate", 40), ("degenerate", 131), ("diagonal", 33), ("kinetic", 60),
         ("random", 384), ("degenerate", 384), ("kinetic", 383), ("random", 440), ("random", 450),
         # the block Jacobi over the whole GPU (n > 512): a padded last block,
         # an odd block count (a padding block), degenerate and Davidson-like
         # spectra, the largest subspace of the 512-band solve
         ("random", 513), ("degenerate", 640), ("kinetic", 1031), ("random", 1536),
         ("kinetic", 1632)]

# bars: (eigenvalue, orthonormality, residual), relative to max |lambda| where scaled
BARS = {"fp64": (1e-12, 1e-12, 1e-11), "mixed": (2e-6, 2e-6, 2e-5)}


def make(kind, n):
    if kind == "random":
        return syn.random_hermitian(n, n) * 3.0
    if kind == "degenerate":
        return degenerate(n, n)
    if kind == "diagonal":
        return np.diag(np.linspace(-1, 4, n)[::-1]).astype(complex)
    # a Davidson-like matrix: large diagonal spread, small coupling
    rng = np.random.default_rng(n)
    H = np.diag(np.sort(rng.uniform(0, 20, n))).astype(complex)
    return H + 1e-3 * syn.random_hermitian(3, n)


@pytest.mark.parametrize("kind,n", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subspace_eigh_vs_lapack(env, kind, n, precision):
    torch, s = env
    H = make(kind, n)
    nk = max(1, n // 3)
    # column-major device layout: row j of the tensor is column j of H
    Ht = torch.from_numpy(np.ascontiguousarray(H.T)).cuda()
    theta, C = s.subspace_eigh(Ht, nk, precision=precision)
    s.sync()
    th = theta.cpu().numpy()
    V = C.cpu().numpy().T           # (n, nk) eigenvectors as columns
    ex = np.linalg.eigvalsh(H)[:nk]
    scale = max(1.0, np.abs(np.linalg.eigvalsh(H)).max())
    be, bo, br = BARS[precision]
    assert np.abs(th - ex).max() <= be * scale, np.abs(th - ex).max()
    assert np.abs(V.conj().T @ V - np.eye(nk)).max() <= bo
    assert np.abs(H @ V - V * th).max() <= br * scale


@pytest.mark.parametrize("kind,m0,n", [("random", 30, 40), ("degenerate", 24, 36),
                                       ("kinetic", 64, 96), ("random", 7, 13),
                                       ("kinetic", 256, 384), ("kinetic", 512, 768),
                                       ("random", 600, 901)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subspace_eigh_warm_start(env, kind, m0, n, precision):
    """Second call on a matrix whose leading m0 x m0 block was diagonalised by the
    first call starts from that eigenbasis (the solver's path between
    Rayleigh-Ritz steps) and must give the same answer as LAPACK."""
    torch, s = env
    if kind == "random":
        H = syn.random_hermitian(n + 1, n) * 3.0
    elif kind == "degenerate":
        H = degenerate(n, n)
    else:
        rng = np.random.default_rng(n)
        H = np.diag(np.sort(rng.uniform(0, 20, n))).astype(complex) + 1e-3 * syn.random_hermitian(5, n)
    Q = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    H0 = np.ascontiguousarray(H[:m0, :m0])
    s.subspace_eigh(torch.from_numpy(np.ascontiguousarray(H0.T)).cuda(), m0 // 2, Q=Q[:m0, :m0].contiguous() if False else None)
    # first call writing Q (ld = n)
    theta0, C0 = s.subspace_eigh(torch.from_numpy(np.ascontiguousarray(H0.T)).cuda(), m0 // 2, Q=Q, warm=0)
    nk = n // 2
    theta, C = s.subspace_eigh(torch.from_numpy(np.ascontiguousarray(H.T)).cuda(), nk, Q=Q, warm=m0,
                               precision=precision)
    s.sync()
    th = theta.cpu().numpy()
    V = C.cpu().numpy().T
    ex = np.linalg.eigvalsh(H)[:nk]
    scale = max(1.0, np.abs(np.linalg.eigvalsh(H)).max())
    be, bo, br = BARS[precision]
    assert np.abs(th - ex).max() <= be * scale, np.abs(th - ex).max()
    assert np.abs(V.conj().T @ V - np.eye(nk)).max() <= bo
    assert np.abs(H @ V - V * th).max() <= br * scale


def _free_electron_rr_matrices():
    """The Rayleigh-Ritz matrices of a block Davidson on free electrons (V = 0,
    no projectors, 12 bands cutting a degenerate shell): near convergence they
    are diagonal up to rounding with exactly degenerate entries, the hard case
    for Jacobi rotations.  Generated with the oracle's Davidson steps."""
    from oracle import davidson as od
    from tests.helpers import case
    cell, b, v, beta, D = case(seed=6, a=7.0, natoms=1, ecut_ry=10.0, lmax=0)
    H = np.diag(b.kinetic).astype(complex)
    nb, m_max, tol = 12, 36, 1e-10
    V = od.cholqr(syn.initial_bands(8, b.npw, nb).T)
    HV = H @ V
    out, valid = [], 0
    for _ in range(40):
        Hs = V.conj().T @ HV
        Hs = 0.5 * (Hs + Hs.conj().T)
        out.append((Hs, valid))
        valid = V.shape[1]
        w, c = np.linalg.eigh(Hs)
        th, c = w[:nb], c[:, :nb]
        X, HX = V @ c, HV @ c
        R = HX - X * th
        rn = np.linalg.norm(R, axis=0)
        if rn.max() <= tol:
            break
        U = np.nonzero(rn > tol)[0]
        T = od.tpa_factor(b.kinetic, X[:, U]) * R[:, U]
        if V.shape[1] + len(U) > m_max:
            V, HV, valid = X, HX, 0
        t0 = np.linalg.norm(T, axis=0)
        for _ in range(2):
            T = T - V @ (V.conj().T @ T)
        T = od.cholqr(T[:, np.linalg.norm(T, axis=0) >= 1e-10 * t0])
        if T.shape[1] == 0:
            V, HV, valid = X, HX, 0
            continue
        V = np.concatenate([V, T], 1)
        HV = np.concatenate([HV, H @ T], 1)
    return out


def test_subspace_eigh_degenerate_davidson_sequence(env):
    torch, s = env
    mats = _free_electron_rr_matrices()
    assert len(mats) > 8
    Q = torch.zeros((36, 36), dtype=torch.complex128, device="cuda")
    for H, warm in mats:
        n, nk = H.shape[0], 12
        Ht = torch.from_numpy(np.ascontiguousarray(H.T)).cuda()
        for w in ((0, warm) if warm else (0,)):
            Qx = Q.clone()
            theta, C = s.subspace_eigh(Ht, nk, Q=Qx, warm=w)
            th = theta.cpu().numpy()
            V = C.cpu().numpy().T
            assert np.abs(th - np.linalg.eigvalsh(H)[:nk]).max() <= 1e-12 * 5
            assert np.abs(V.conj().T @ V - np.eye(nk)).max() <= 1e-12
        s.subspace_eigh(Ht, nk, Q=Q, warm=warm)
    s.sync()


# ------------------------------------------------------------ Cholesky-QR
@pytest.mark.parametrize("k", [100, 200, 300, 545, 1024])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subspace_cholqr_paths(env, k, precision):
    """The orthonormalisation factor on one block (k <= 156 FP64 / 221 FP32)
    and blocked over the whole GPU (above), with one column below the drop
    threshold (and, in FP64, two dependent columns): the kept count is the rank,
    T Tr is orthonormal, and without drops Tr equals D^-1/2 L^-H from LAPACK's
    Cholesky of the unit-diagonal Gram matrix."""
    torch, s = env
    rng = np.random.default_rng(k)
    n = 2 * k + 400
    T = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    # exactly dependent columns: dropped by the FP64 pivot test (in FP32 the
    # rounding of a late pivot can exceed its threshold, so only the norm-based
    # drop is required there)
    dep = [(17, 3), (k - 5, 40)] if precision == "fp64" else []
    for c, src in dep:
        T[:, c] = (0.3 - 0.7j) * T[:, src] + 1e-15 * rng.standard_normal(n)
    T[:, 11] *= 1e-12
    t0 = np.linalg.norm(T, axis=0)
    t0[11] = 1.0
    S = T.conj().T @ T
    Tr, kept = s.cholqr(torch.from_numpy(S.T.copy()).cuda(), torch.from_numpy(t0).cuda(),
                        1e-10, precision)
    assert kept == k - 1 - len(dep)
    Q = T @ Tr.cpu().numpy().T[:, :kept]
    # FP32: forward error about kappa sqrt(k) eps32 (kappa of the Gram matrix
    # up to 22 here): 1e-3
    tol = 1e-10 if precision == "fp64" else 1e-3
    assert np.abs(Q.conj().T @ Q - np.eye(kept)).max() <= tol
    assert np.abs(Tr.cpu().numpy().T[:, kept:]).max() == 0.0
    # no drops: the factor itself against LAPACK
    T2 = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    S2 = T2.conj().T @ T2
    Tr2, kept2 = s.cholqr(torch.from_numpy(S2.T.copy()).cuda(), None, 0.0, precision)
    assert kept2 == k
    dinv = 1.0 / np.sqrt(S2.diagonal().real)
    L = np.linalg.cholesky(S2 * dinv[:, None] * dinv[None, :])
    ref = dinv[:, None] * np.linalg.inv(L).conj().T
    err = np.abs(Tr2.cpu().numpy().T - ref).max() / np.abs(ref).max()
    assert err <= (1e-11 if precision == "fp64" else 1e-3), err
