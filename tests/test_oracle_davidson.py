"""Pins of the oracle's block Davidson (CPU only): brute-force diagonalisation,
the variational principle, residual bounds and independence of the
preconditioner."""
import numpy as np
import pytest

from oracle import basis as ob
from oracle import davidson as od
from oracle import hamiltonian as oh
from paper_1709_10010_gb300 import synthetic as syn


def setup(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1, k=(0, 0, 0)):
    cell = syn.make_cell(seed, a, natoms, ecut_ry, lmax, kpoint=k)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    return cell, b, v, beta, D


@pytest.mark.parametrize("k", [(0, 0, 0), (0.25, 0.25, -0.25)])
def test_davidson_matches_dense_eigh(k):
    cell, b, v, beta, D = setup(k=k)
    nb = 8
    H = oh.dense_h(b, v, beta, D)
    ex = np.linalg.eigvalsh(H)[:nb]
    X0 = syn.initial_bands(1, b.npw, nb).T
    res = od.davidson(lambda X: H @ X, b.kinetic, X0, nb, tol=1e-10)
    assert res.converged
    np.testing.assert_allclose(res.eig, ex, rtol=0, atol=1e-10)
    # variational: Ritz values never fall below the exact ones
    assert np.all(res.eig >= ex - 1e-12)
    # the returned vectors are orthonormal eigenvectors within the residual bound
    assert np.abs(res.X.conj().T @ res.X - np.eye(nb)).max() < 1e-12
    assert np.linalg.norm(H @ res.X - res.X * res.eig, axis=0).max() <= 1e-10


def test_davidson_uses_fft_operator_and_any_preconditioner():
    cell, b, v, beta, D = setup(seed=3, natoms=3, lmax=2)
    nb = 6
    ex = np.linalg.eigvalsh(oh.dense_h(b, v, beta, D))[:nb]
    X0 = syn.initial_bands(2, b.npw, nb).T

    def apply(X):
        return oh.apply_h(b, v, beta, D, X.T).T
    r1 = od.davidson(apply, b.kinetic, X0, nb, tol=1e-9, precond="tpa")
    r2 = od.davidson(apply, b.kinetic, X0, nb, tol=1e-9, precond="none", max_iter=400)
    np.testing.assert_allclose(r1.eig, ex, atol=1e-9)
    np.testing.assert_allclose(r2.eig, ex, atol=1e-9)
    assert r1.iters < r2.iters        # TPA helps


def test_residual_bound_holds_midway():
    """Bauer-Fike / Weyl: each Ritz value lies within ||r_n|| of an exact eigenvalue."""
    cell, b, v, beta, D = setup(seed=4)
    H = oh.dense_h(b, v, beta, D)
    ev = np.linalg.eigvalsh(H)
    nb = 5
    X0 = syn.initial_bands(3, b.npw, nb).T
    seen = []

    def hook(it, X, theta, R):
        rn = np.linalg.norm(R, axis=0)
        for t, r in zip(theta, rn):
            seen.append(np.min(np.abs(ev - t)) <= r + 1e-12)
    od.davidson(lambda X: H @ X, b.kinetic, X0, nb, tol=1e-8, max_iter=6, hook=hook)
    assert seen and all(seen)


def test_tpa_factor_limits():
    """K(0) = 1, K decreasing, and K(x) ~ 1/(2x) for large x = T_G/E_ref, with
    E_ref = <x|T|x> the band's kinetic energy (here 0.5)."""
    T = np.array([0.0, 1.0, 1e4, 3.0])
    X = np.array([[1.0], [1.0], [0.0], [0.0]], dtype=complex) / np.sqrt(2)
    K = od.tpa_factor(T, X)[:, 0]
    assert abs(K[0] - 1.0) < 1e-15
    x = T / 0.5
    assert abs(K[2] * 2 * x[2] - 1.0) < 1e-3
    assert K[0] > K[1] > K[3] > K[2]
    # at x = 1 the published rational function gives 65/81
    T1 = np.array([0.5, 0.5])
    X1 = np.array([[1.0], [1.0]], dtype=complex) / np.sqrt(2)
    assert abs(od.tpa_factor(T1, X1)[0, 0] - 65.0 / 81.0) < 1e-15


def test_cholqr_drops_dependent_columns():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((50, 3)) + 1j * rng.standard_normal((50, 3))
    T = np.concatenate([A, A[:, :1] * 2.0], axis=1)
    Q = od.cholqr(T)
    assert Q.shape[1] == 3
    assert np.abs(Q.conj().T @ Q - np.eye(3)).max() < 1e-13
