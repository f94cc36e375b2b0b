"""Block Davidson eigensolver of the oracle (TEST INFRASTRUCTURE; see
``oracle/__init__``).

The paper names "a Davidson-like algorithm [Davidson 1975]" (Sec. "Dynamic
perturbations ... spectroscopies", optical absorption) and the subspace
diagonalisation of the iterative diagonalisation in PWscf (Sec. "New
parallelization levels", the O_ij = <psi_i|O|psi_j> matrices) without writing
the algorithm out.  This is the textbook block Davidson for the lowest ``nb``
eigenpairs of a Hermitian operator, step by step:

1. X0 = starting bands, orthonormalised by Cholesky-QR (twice); V = X0, HV = H X0.
2. Each iteration: Hs = V^H HV, Hermitised (Hs + Hs^H)/2; its lowest nb
   eigenpairs (theta, c), ascending; X = V c, HX = HV c, R = HX - X diag(theta).
3. Converged when ||r_n||_2 <= tol for every band n < nb.
4. For the unconverged bands, t_n = K_n (.) r_n with the Teter-Payne-Allan
   preconditioner K (Teter, Payne, Allan, Phys. Rev. B 40, 12255 (1989)),
   its reference energy the kinetic energy <x_n|T|x_n> of the Ritz vector.
5. If the subspace would exceed m_max columns, restart with V = X, HV = HX.
6. Project T against V twice (classical Gram-Schmidt), drop columns whose norm
   fell below 1e-10 of the norm before projection, orthonormalise by Cholesky-QR
   (twice; a column whose Cholesky pivot falls below 1e-12 of its unit norm is
   dropped), then V <- [V T], HV <- [HV, H T].

Vectors are columns of (npw, m) arrays here.  The small Hermitian eigenproblem
and the Cholesky factor use numpy/LAPACK as library steps.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def tpa_factor(kinetic: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Teter-Payne-Allan diagonal K for the bands X (npw, k), unit norm.

    x = T_G / E_ref with E_ref = <x_n|T|x_n>/<x_n|x_n> the kinetic energy of the
    band being corrected (the reference energy of the published method), and
    K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4)."""
    w = np.abs(X) ** 2
    eref = (kinetic[:, None] * w).sum(axis=0) / w.sum(axis=0)
    x = kinetic[:, None] / eref[None, :]
    p = 27.0 + 18.0 * x + 12.0 * x ** 2 + 8.0 * x ** 3
    return p / (p + 16.0 * x ** 4)


def cholesky_drop(S: np.ndarray, drop_tol: float = 1e-12):
    """Cholesky S = L L^H of a Hermitian matrix with unit-ish diagonal, dropping
    any column whose pivot falls below ``drop_tol``.  Returns (L, kept indices)."""
    keep = list(range(S.shape[0]))
    while True:
        Sk = S[np.ix_(keep, keep)]
        n = len(keep)
        L = np.zeros_like(Sk)
        bad = -1
        for j in range(n):
            d = Sk[j, j].real - np.sum(np.abs(L[j, :j]) ** 2)
            if d <= drop_tol:
                bad = j
                break
            L[j, j] = np.sqrt(d)
            for i in range(j + 1, n):
                L[i, j] = (Sk[i, j] - L[i, :j] @ np.conj(L[j, :j])) / L[j, j]
        if bad < 0:
            return L, keep
        keep.pop(bad)


def cholqr(T: np.ndarray):
    """Orthonormalise the columns of T (npw, k) by Cholesky-QR, twice, dropping
    dependent columns.  Returns the orthonormal columns."""
    for _ in range(2):
        if T.shape[1] == 0:
            return T
        nrm = np.linalg.norm(T, axis=0)
        T = T / nrm[None, :]
        S = T.conj().T @ T
        L, keep = cholesky_drop(S)
        T = T[:, keep]
        T = T @ np.linalg.inv(L).conj().T       # T L^{-H}: (T L^-H)^H (T L^-H) = I
    return T


@dataclasses.dataclass
class DavidsonResult:
    eig: np.ndarray
    X: np.ndarray          # (npw, nb) eigenvector columns
    resid: np.ndarray      # (nb,) final residual norms
    iters: int
    n_apply: int
    converged: bool
    history: list          # max residual after each iteration


def davidson(apply_h, kinetic, X0, nb, tol=1e-10, max_iter=200, m_max=None,
             precond="tpa", hook=None) -> DavidsonResult:
    """Lowest ``nb`` eigenpairs of the Hermitian operator ``apply_h``.

    ``apply_h`` maps (npw, k) columns to (npw, k) columns.  ``X0`` is (npw, nb).
    ``precond`` is "tpa" or "none".  ``hook(it, X, theta, R)`` (optional) sees the
    Ritz pairs and residuals of every iteration (used to build training data)."""
    m_max = 4 * nb if m_max is None else int(m_max)
    V = cholqr(np.array(X0, dtype=np.complex128))
    HV = apply_h(V)
    n_apply = V.shape[1]
    history = []
    it = 0
    while True:
        it += 1
        Hs = V.conj().T @ HV
        Hs = 0.5 * (Hs + Hs.conj().T)
        w, c = np.linalg.eigh(Hs)
        theta, c = w[:nb], c[:, :nb]
        X = V @ c
        HX = HV @ c
        R = HX - X * theta[None, :]
        rn = np.linalg.norm(R, axis=0)
        history.append(float(rn.max()))
        if hook is not None:
            hook(it, X, theta, R)
        if rn.max() <= tol or it >= max_iter:
            return DavidsonResult(eig=theta, X=X, resid=rn, iters=it, n_apply=n_apply,
                                  converged=bool(rn.max() <= tol), history=history)
        U = np.nonzero(rn > tol)[0]
        Ru = R[:, U]
        T = tpa_factor(kinetic, X[:, U]) * Ru if precond == "tpa" else Ru.copy()
        if V.shape[1] + len(U) > m_max:
            V, HV = X, HX
        t0 = np.linalg.norm(T, axis=0)
        for _ in range(2):
            T = T - V @ (V.conj().T @ T)
        keep = np.linalg.norm(T, axis=0) >= 1e-10 * t0
        T = cholqr(T[:, keep])
        if T.shape[1] == 0:
            V, HV = X, HX
            continue
        HT = apply_h(T)
        n_apply += T.shape[1]
        V = np.concatenate([V, T], axis=1)
        HV = np.concatenate([HV, HT], axis=1)
