"""H|psi> of the oracle (TEST INFRASTRUCTURE; see ``oracle/__init__``).

The operator is the norm-conserving reduction (overlap S = 1) of the Kohn-Sham
Hamiltonian of Eq. pauli_ks (Sec. "Fully relativistic projector augmented-wave
method"): kinetic energy p^2/2m acting on the FFT mesh, the local potential
V_LOC(r), and the separable nonlocal term sum_{mn} D_mn |beta_m><beta_n|.  In a
plane-wave basis, Hartree atomic units:

    (H psi)_G = 1/2 |k+G|^2 psi_G
              + sum_{G' in sphere} Vt(G - G') psi_{G'}
              + sum_{i,j} beta_i(G) D_ij sum_{G'} conj(beta_j(G')) psi_{G'}

with Vt(g) = N^-3 sum_r V(r) exp(-i g.r) the discrete Fourier transform of the
potential sampled on the N1 x N2 x N3 grid, g taken modulo N per axis.  The
projector products becp = beta^H psi are the p_ij of Sec. "New parallelization
levels".

Array conventions: psi is (nb, npw) (row = band), beta is (P, npw) (row =
projector), D is (P,) for a diagonal or (P, P) Hermitian, v_r is (N1, N2, N3)
C order.  Two independent routes compute the local term:

* ``local_dense``  the plain definition: an explicit circulant matrix Vt(G-G');
* ``local_fft``    scatter to the box, inverse 3D FFT (exp(+iG.r), unscaled),
                   multiply by V(r), forward 3D FFT (exp(-iG.r), times N^-3),
                   gather — the route of the FFT mesh the paper describes.
"""
from __future__ import annotations

import numpy as np


def v_tilde(v_r: np.ndarray) -> np.ndarray:
    """Vt(m) = N^-3 sum_j V(r_j) exp(-2 pi i m.j/N), indexed by m mod N."""
    return np.fft.fftn(v_r) / v_r.size


def local_matrix(miller: np.ndarray, fft, v_r: np.ndarray) -> np.ndarray:
    """Dense npw x npw matrix Vt(G - G') (Hermitian for real V)."""
    vt = v_tilde(v_r)
    d = miller[:, None, :] - miller[None, :, :]
    return vt[d[..., 0] % fft[0], d[..., 1] % fft[1], d[..., 2] % fft[2]]


def local_dense(miller, fft, v_r, psi) -> np.ndarray:
    """Local term by the plain definition, in row blocks to bound memory."""
    psi = np.atleast_2d(psi)
    vt = v_tilde(v_r)
    out = np.zeros_like(psi, dtype=np.complex128)
    npw = miller.shape[0]
    step = max(1, int(2 ** 24 // max(npw, 1)))
    for g0 in range(0, npw, step):
        d = miller[g0:g0 + step, None, :] - miller[None, :, :]
        vmat = vt[d[..., 0] % fft[0], d[..., 1] % fft[1], d[..., 2] % fft[2]]
        out[:, g0:g0 + step] = psi @ vmat.T
    return out


def local_fft(miller, fft, v_r, psi) -> np.ndarray:
    """Local term by scatter / inverse FFT / multiply / forward FFT / gather."""
    psi = np.atleast_2d(psi)
    n1, n2, n3 = fft
    idx = (miller[:, 0] % n1, miller[:, 1] % n2, miller[:, 2] % n3)
    ntot = n1 * n2 * n3
    out = np.empty_like(psi, dtype=np.complex128)
    for b in range(psi.shape[0]):
        box = np.zeros((n1, n2, n3), dtype=np.complex128)
        box[idx] = psi[b]
        psi_r = np.fft.ifftn(box) * ntot        # sum_G c_G exp(+iG.r)
        prod = v_r * psi_r
        back = np.fft.fftn(prod) / ntot         # N^-3 sum_r f(r) exp(-iG.r)
        out[b] = back[idx]
    return out


def _d_matrix(D) -> np.ndarray:
    D = np.asarray(D)
    return np.diag(D.astype(np.complex128)) if D.ndim == 1 else D.astype(np.complex128)


def becp(beta, psi) -> np.ndarray:
    """p = beta^H psi as a (P, nb) array: p[j, b] = sum_G conj(beta_j(G)) psi_b(G)."""
    return np.conj(beta) @ np.atleast_2d(psi).T


def nonlocal_term(beta, D, psi) -> np.ndarray:
    """sum_ij beta_i D_ij <beta_j|psi>, returned as (nb, npw)."""
    if beta is None or beta.shape[0] == 0:
        return np.zeros_like(np.atleast_2d(psi), dtype=np.complex128)
    p = becp(beta, psi)
    return (beta.T @ (_d_matrix(D) @ p)).T


def apply_h(basis, v_r, beta, D, psi, route: str = "fft") -> np.ndarray:
    """(H psi) for every band; ``route`` is "fft" or "dense" for the local term."""
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    loc = (local_fft if route == "fft" else local_dense)(basis.miller, basis.fft, v_r, psi)
    return basis.kinetic[None, :] * psi + loc + nonlocal_term(beta, D, psi)


def dense_h(basis, v_r, beta, D) -> np.ndarray:
    """The explicit npw x npw matrix H_{GG'} (for brute-force diagonalisation)."""
    h = local_matrix(basis.miller, basis.fft, v_r)
    h[np.diag_indices_from(h)] += basis.kinetic
    if beta is not None and beta.shape[0]:
        h += beta.T @ _d_matrix(D) @ np.conj(beta)
    return h
