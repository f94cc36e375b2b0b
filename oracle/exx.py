"""Exact (Fock) exchange and its adaptively compressed form (TEST
INFRASTRUCTURE; see ``oracle/__init__``).

Sec. "Advanced implementation of exact (Fock) exchange and hybrid functionals":
the Fock operator of Eq. Vx acting on a band phi, with the pair densities and
their potentials of Eq. Poisson solved in reciprocal space, and the adaptively
compressed exchange (ACE) operator of Eq. Vxace.  Hartree atomic units (e = 1).

* exchange   (V_x phi)(r) = - sum_j f_j psi_j(r) v_j(r),
             v_j(r) = int rho_j(r') / |r - r'| dr',  rho_j(r) = conj(psi_j(r)) phi(r),
             for occupied bands psi_j with weights f_j (all at the system's k,
             so that rho_j is periodic).  Route: every band on the FFT grid
             (scatter, inverse FFT), rho_j on the grid, its grid DFT rho_j(G),
             v_j(G) = 4 pi rho_j(G) / |G|^2 for G != 0 and v_j(0) = 0 (the
             divergent G = 0 term is left out, as the neutralising background
             of the Hartree potential), back to the grid, the product with
             psi_j, forward FFT, gather on the sphere.  On a box with
             N_d >= 4 mmax_d + 1 every step is exact: rho_j has Miller indices
             within +-2 mmax_d and the product psi_j v_j within +-3 mmax_d,
             which cannot alias onto the sphere (|m_d| <= mmax_d < N_d - 3 mmax_d).
* exchange_brute  the same operator as one sum in reciprocal space, with no FFT:
             (V_x phi)(g) = -(4 pi / Omega) sum_j f_j
                 sum_{a, b in sphere, a != b, g - b + a in sphere}
                     c_j(g - b + a) conj(c_j(a)) d(b) / |b - a|^2
             (c_j, d the coefficients of psi_j and phi).
* ace        xi_i = V_x psi_i, M = <psi_j | xi_m>, and V_ACE phi =
             sum_jm xi_j (M^-1)_jm <xi_m | phi> (Eq. Vxace), written as
             V_ACE = -zeta zeta^H with -M = L L^H (Cholesky) and
             zeta = xi L^-H; alpha scales it (the exchange fraction of a hybrid
             functional).

Band arrays are (nb, npw) complex (row = band) in the order of ``basis.miller``.
"""
from __future__ import annotations

import numpy as np

from .basis import reciprocal


def coulomb_kernel(lattice, fft) -> np.ndarray:
    """4 pi / |G|^2 on the FFT grid (index m_d read as m_d - N_d above N_d / 2),
    0 at G = 0."""
    b = reciprocal(lattice)
    ms = []
    for d, n in enumerate(fft):
        m = np.arange(n)
        m = np.where(m > n // 2, m - n, m)
        shape = [1, 1, 1]
        shape[d] = n
        ms.append(m.reshape(shape))
    gx = ms[0] * b[0, 0] + ms[1] * b[1, 0] + ms[2] * b[2, 0]
    gy = ms[0] * b[0, 1] + ms[1] * b[1, 1] + ms[2] * b[2, 1]
    gz = ms[0] * b[0, 2] + ms[1] * b[1, 2] + ms[2] * b[2, 2]
    g2 = gx ** 2 + gy ** 2 + gz ** 2
    return np.where(g2 > 0, 4.0 * np.pi / np.where(g2 > 0, g2, 1.0), 0.0)


def _to_grid(miller, fft, c) -> np.ndarray:
    """sum_G c(G) exp(i G.r) on the grid (the periodic part times Omega^1/2)."""
    n1, n2, n3 = fft
    box = np.zeros(tuple(fft), dtype=np.complex128)
    box[miller[:, 0] % n1, miller[:, 1] % n2, miller[:, 2] % n3] = c
    return np.fft.ifftn(box) * box.size


def _from_grid(miller, fft, w) -> np.ndarray:
    """Coefficients on the sphere of the grid function w: N^-3 sum_r w e^{-iG.r}."""
    n1, n2, n3 = fft
    wg = np.fft.fftn(w) / w.size
    return wg[miller[:, 0] % n1, miller[:, 1] % n2, miller[:, 2] % n3]


def exchange(basis, lattice, psi_occ, occ, phi) -> np.ndarray:
    """V_x phi for the bands phi (nb, npw), occupied bands psi_occ (nocc, npw)
    with weights occ (nocc,), by the FFT route."""
    miller, fft = np.asarray(basis.miller), tuple(basis.fft)
    volume = abs(np.linalg.det(np.asarray(lattice, dtype=np.float64)))
    kern = coulomb_kernel(lattice, fft)
    psi_occ, phi = np.atleast_2d(psi_occ), np.atleast_2d(phi)
    u = [_to_grid(miller, fft, c) for c in psi_occ]       # Omega^1/2 psi_j(r) e^{-ik.r}
    out = np.zeros_like(phi, dtype=np.complex128)
    for i, d in enumerate(phi):
        p = _to_grid(miller, fft, d)
        w = np.zeros(tuple(fft), dtype=np.complex128)
        for j, uj in enumerate(u):
            rho_g = np.fft.fftn(np.conj(uj) * p) / p.size / volume   # rho_j(G)
            v = np.fft.ifftn(kern * rho_g) * p.size                    # v_j(r)
            w -= occ[j] * uj * v
        out[i] = _from_grid(miller, fft, w)
    return out


def exchange_brute(basis, lattice, psi_occ, occ, phi) -> np.ndarray:
    """V_x phi by the reciprocal-space sum, no FFT (small spheres only)."""
    miller = np.asarray(basis.miller)
    npw = miller.shape[0]
    volume = abs(np.linalg.det(np.asarray(lattice, dtype=np.float64)))
    b = reciprocal(lattice)
    where = {tuple(m): i for i, m in enumerate(miller.tolist())}
    psi_occ, phi = np.atleast_2d(psi_occ), np.atleast_2d(phi)
    # q = b - a over all pairs (a, b) of the sphere, and its Coulomb factor
    dq = miller[None, :, :] - miller[:, None, :]              # [a, b] -> b - a
    qc = dq @ b
    q2 = np.einsum("abk,abk->ab", qc, qc)
    fac = np.where(q2 > 0, 4.0 * np.pi / np.where(q2 > 0, q2, 1.0), 0.0)
    out = np.zeros_like(phi, dtype=np.complex128)
    for gi in range(npw):
        # a' = g - b + a must lie in the sphere
        src = miller[gi][None, None, :] - dq                  # [a, b] -> g - (b - a)
        idx = np.array([[where.get(tuple(s), -1) for s in row] for row in src.tolist()])
        ok = (idx >= 0) & (fac > 0)
        for j in range(psi_occ.shape[0]):
            cj = psi_occ[j]
            t = np.where(ok, cj[np.where(ok, idx, 0)] * fac, 0.0) * np.conj(cj)[:, None]
            out[:, gi] -= occ[j] * (phi @ t.sum(axis=0))
    return out / volume


def ace(basis, lattice, psi_occ, occ, alpha=1.0) -> np.ndarray:
    """zeta (nocc, npw) with V_ACE = -zeta^H-outer: V_ACE phi = -sum_k zeta_k <zeta_k|phi>."""
    psi_occ = np.atleast_2d(psi_occ)
    xi = exchange(basis, lattice, psi_occ, occ, psi_occ)     # rows xi_i = V_x psi_i
    M = np.conj(psi_occ) @ xi.T                              # M[j, m] = <psi_j | xi_m>
    M = 0.5 * (M + M.conj().T)
    L = np.linalg.cholesky(-M)                               # -M = L L^H
    # zeta = xi L^-H as columns: zeta_cols = xi_cols @ inv(L)^H
    zeta_cols = xi.T @ np.linalg.inv(L).conj().T
    return np.sqrt(alpha) * zeta_cols.T


def apply_ace(zeta, phi) -> np.ndarray:
    """V_ACE phi = -zeta (zeta^H phi) for bands phi (nb, npw)."""
    phi = np.atleast_2d(phi)
    return -(np.conj(zeta) @ phi.T).T @ zeta
