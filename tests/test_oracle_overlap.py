"""Pins of the oracle's generalised eigenproblem (CPU only): S by its
definition against its dense matrix; a single projector (closed forms of S and
S^-1/2 on it); the separable S^-1/2 against the dense inverse square root; the
LAPACK generalised pairs against the Loewdin-transformed standard problem and,
for q = 0, against the standard one; S-orthonormal eigenvectors with zero
residual H x - e S x."""
import numpy as np
import scipy.linalg

from oracle import hamiltonian as oh
from oracle import overlap as oo
from paper_1709_10010_gb300 import synthetic as syn
from tests.helpers import case


def q_matrix(P, seed, full=False):
    rng = np.random.default_rng(seed)
    if not full:
        return rng.uniform(0.1, 0.8, P)
    a = 0.2 * (rng.standard_normal((P, P)) + 1j * rng.standard_normal((P, P)))
    return 0.5 * (a + a.conj().T) + np.eye(P)


def test_apply_s_matches_dense():
    cell, b, v, beta, D = case(seed=0, a=7.0, natoms=3, ecut_ry=10.0, lmax=1)
    for full in (False, True):
        q = q_matrix(beta.shape[0], 1, full)
        S = oo.dense_s(beta, q, b.npw)
        assert np.abs(S - S.conj().T).max() <= 1e-14 * np.abs(S).max()
        assert np.linalg.eigvalsh(S).min() > 0.5
        psi = syn.initial_bands(2, b.npw, 3)
        np.testing.assert_allclose(oo.apply_s(beta, q, psi), psi @ S.T, rtol=0, atol=1e-12)


def test_single_projector_closed_forms():
    cell, b, v, beta, D = case(seed=1, a=7.0, natoms=1, ecut_ry=10.0, lmax=0)
    beta = beta[:1]
    q = np.array([0.7])
    nrm2 = float(np.vdot(beta[0], beta[0]).real)
    np.testing.assert_allclose(oo.apply_s(beta, q, beta), (1 + 0.7 * nrm2) * beta, rtol=1e-13)
    K = oo.s_inv_sqrt_coef(beta, q)
    np.testing.assert_allclose(oo.apply_s_inv_sqrt(beta, K, beta), (1 + 0.7 * nrm2) ** -0.5 * beta,
                               rtol=1e-12)
    # and the complement of the projector is left alone
    psi = syn.initial_bands(3, b.npw, 1)
    perp = psi - (np.vdot(beta[0], psi[0]) / nrm2) * beta
    np.testing.assert_allclose(oo.apply_s_inv_sqrt(beta, K, perp), perp, rtol=0, atol=1e-14)


def test_separable_inverse_square_root_matches_dense():
    # a shifted k: the projector Gram matrix is complex (at k = 0 it is real)
    cell, b, v, beta, D = case(seed=2, a=7.0, natoms=3, ecut_ry=10.0, lmax=1, k=(0.25, -0.1, 0.3))
    G = np.conj(beta) @ beta.T
    assert np.abs(G.imag).max() > 1e-3 * np.abs(G).max()
    for full in (False, True):
        q = q_matrix(beta.shape[0], 3, full)
        S = oo.dense_s(beta, q, b.npw)
        w, U = np.linalg.eigh(S)
        Sm = (U * w ** -0.5) @ U.conj().T
        K = oo.s_inv_sqrt_coef(beta, q)
        psi = syn.initial_bands(4, b.npw, 5)
        np.testing.assert_allclose(oo.apply_s_inv_sqrt(beta, K, psi), psi @ Sm.T, rtol=0, atol=1e-12)
        X = oo.apply_s_inv_sqrt(beta, K, np.eye(b.npw))        # rows: S^-1/2 e_g
        np.testing.assert_allclose(X.conj() @ S @ X.T, np.eye(b.npw), rtol=0, atol=1e-12)


def test_generalised_pairs():
    cell, b, v, beta, D = case(seed=3, a=7.5, natoms=3, ecut_ry=10.0, lmax=1, k=(0.1, 0.2, -0.3))
    H = oh.dense_h(b, v, beta, D)
    q = q_matrix(beta.shape[0], 5, True)
    S = oo.dense_s(beta, q, b.npw)
    e, X = oo.gen_eigh(H, S, 8)
    # Loewdin: the standard problem of S^-1/2 H S^-1/2 has the same spectrum
    w, U = np.linalg.eigh(S)
    Sm = (U * w ** -0.5) @ U.conj().T
    np.testing.assert_allclose(np.linalg.eigvalsh(Sm @ H @ Sm)[:8], e, rtol=0, atol=1e-11)
    np.testing.assert_allclose(X.conj() @ S @ X.T, np.eye(8), rtol=0, atol=1e-11)
    R = X @ H.T - e[:, None] * (X @ S.T)
    assert np.abs(R).max() <= 1e-10
    # q = 0 is the standard problem
    e0, _ = oo.gen_eigh(H, oo.dense_s(beta, np.zeros(beta.shape[0]), b.npw), 8)
    np.testing.assert_allclose(e0, np.linalg.eigvalsh(H)[:8], rtol=0, atol=1e-11)
