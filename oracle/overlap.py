"""The generalised eigenproblem of ultrasoft / PAW projectors (TEST
INFRASTRUCTURE; see ``oracle/__init__``).

Eq. pauli_ks (Sec. "Fully relativistic projector augmented-wave method")
carries the overlap operator S: the Kohn-Sham equations read
H psi = epsilon S psi.  The paper refers its definition to the literature; the
separable form over the same projectors as the nonlocal term is taken here,

    S = 1 + sum_ij |beta_i> q_ij <beta_j|,   q Hermitian, S positive definite,

so that S psi = psi + beta (q (beta^H psi)).  Band arrays are (nb, npw)
(row = band), beta is (P, npw), q is (P,) for a diagonal or (P, P).

* apply_s        S psi by its definition.
* dense_s        the npw x npw matrix of S.
* gen_eigh       the lowest pairs of H x = e S x by LAPACK's Hermitian-definite
                 generalised solver (scipy.linalg.eigh(H, S)); eigenvectors
                 S-orthonormal.
* s_inv_sqrt_coef  the P x P matrix K with S^-1/2 = 1 + beta^H-outer K: from
                 G = beta beta^H = W diag(g) W^H (kept g > 1e-12 max g),
                 M = g^1/2 W^H q W g^1/2 = U diag(mu) U^H, and
                 K = W g^-1/2 U diag((1 + mu)^-1/2 - 1) U^H g^-1/2 W^H,
                 the square-root inverse of S restricted to the span of the
                 projectors (S is the identity on its complement).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .hamiltonian import _d_matrix, nonlocal_term


def apply_s(beta, q, psi) -> np.ndarray:
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    return psi + nonlocal_term(beta, q, psi)


def dense_s(beta, q, npw) -> np.ndarray:
    s = np.eye(npw, dtype=np.complex128)
    if beta is not None and beta.shape[0]:
        s += beta.T @ _d_matrix(q) @ np.conj(beta)
    return s


def gen_eigh(H, S, nb):
    """Lowest nb eigenvalues and S-orthonormal eigenvectors (rows) of H x = e S x."""
    w, v = scipy.linalg.eigh(H, S, subset_by_index=[0, nb - 1])
    return w, v.T


def s_inv_sqrt_coef(beta, q) -> np.ndarray:
    """K (P x P) with S^-1/2 psi = psi + beta^T K conj(beta) psi (rows)."""
    Q = _d_matrix(q)
    G = np.conj(beta) @ beta.T                  # G[i, j] = <beta_i | beta_j>
    g, W = np.linalg.eigh(0.5 * (G + G.conj().T))
    keep = g > 1e-12 * g.max()
    g, W = g[keep], W[:, keep]
    sq = np.sqrt(g)
    # S on span(beta) in the orthonormal basis u = beta^T W g^-1/2 (columns):
    # beta^T = u g^1/2 W^H, so S = 1 + u M u^H with M = g^1/2 W^H q W g^1/2
    M = (sq[:, None] * (W.conj().T @ Q @ W)) * sq[None, :]
    M = 0.5 * (M + M.conj().T)
    mu, U = np.linalg.eigh(M)
    if mu.min() <= -1.0:
        raise ValueError("S is not positive definite")
    F = (U * ((1.0 + mu) ** -0.5 - 1.0)[None, :]) @ U.conj().T
    Winv = W / sq[None, :]                      # W g^-1/2
    return Winv @ F @ Winv.conj().T


def apply_s_inv_sqrt(beta, K, psi) -> np.ndarray:
    """S^-1/2 psi = psi + sum_ij beta_i K_ij <beta_j|psi>."""
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    return psi + nonlocal_term(beta, K, psi)
