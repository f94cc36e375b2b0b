"""The self-consistent-field steps either side of H|psi> (TEST INFRASTRUCTURE;
see ``oracle/__init__``): the electron density of a set of bands, the Hartree
potential by the Fourier-space Poisson solution, and the local-density
exchange-correlation potential, whose sum with the ionic potential is the new
V_LOC(r) of the Kohn-Sham Hamiltonian (Sec. "Introduction": the Kohn-Sham
equations solved self-consistently; the Hartree term of exact exchange, Sec.
"Advanced implementation of exact (Fock) exchange", is the same Poisson
solution applied to pair densities).  Hartree atomic units.

Grids are N1 x N2 x N3 arrays in C order; grid point (i1, i2, i3) is
r = sum_d (i_d / N_d) a_d.

* density   rho(r) = sum_n f_n |psi_n(r)|^2 with
            psi_n(r) = Omega^{-1/2} sum_G c_n(G) exp(i (k+G).r)
            (the phase exp(i k.r) has modulus one and drops out).
* hartree   rho(r) = sum_G rho(G) exp(i G.r) on the grid; V_H(G) =
            4 pi rho(G) / |G|^2 for G != 0, V_H(G = 0) = 0 (a neutralising
            background), and G on a Nyquist plane (m_d = N_d / 2 for even N_d)
            dropped as well (its sign is ambiguous; a density made of bands in
            the sphere has no such component when N_d >= 4 mmax_d + 1).
            E_H = (1/2) int V_H rho dr = (Omega / 2) sum_G 4 pi |rho(G)|^2/|G|^2.
* lda_xc    Slater exchange, eps_x = -(3/4) (3 rho / pi)^(1/3), v_x = 4/3 eps_x,
            and the Perdew-Zunger parametrisation (Phys. Rev. B 23, 5048, 1981)
            of the Ceperley-Alder correlation energy of the unpolarised
            electron gas, r_s = (3 / (4 pi rho))^(1/3):
              r_s >= 1: eps_c = g / (1 + b1 sqrt(r_s) + b2 r_s),
                        v_c = eps_c (1 + 7/6 b1 sqrt(r_s) + 4/3 b2 r_s)
                                    / (1 + b1 sqrt(r_s) + b2 r_s)
              r_s < 1:  eps_c = A ln r_s + B + C r_s ln r_s + D r_s,
                        v_c = A ln r_s + (B - A/3) + 2/3 C r_s ln r_s
                              + (2 D - C)/3 r_s
            with g = -0.1423, b1 = 1.0529, b2 = 0.3334, A = 0.0311,
            B = -0.048, C = 0.0020, D = -0.0116.  Points with rho below
            RHO_MIN get eps_xc = v_xc = 0.
"""
from __future__ import annotations

import numpy as np

from .basis import reciprocal

PZ = dict(g=-0.1423, b1=1.0529, b2=0.3334, A=0.0311, B=-0.048, C=0.0020, D=-0.0116)
RHO_MIN = 1e-20


def density(miller, fft, psi, occ, volume) -> np.ndarray:
    """rho on the grid from bands psi (nb, npw) with Miller rows (npw, 3) and
    occupations occ (nb,)."""
    n1, n2, n3 = fft
    idx = (np.asarray(miller)[:, 0] % n1, np.asarray(miller)[:, 1] % n2, np.asarray(miller)[:, 2] % n3)
    ntot = n1 * n2 * n3
    rho = np.zeros((n1, n2, n3))
    for b in range(np.atleast_2d(psi).shape[0]):
        box = np.zeros((n1, n2, n3), dtype=np.complex128)
        box[idx] = np.atleast_2d(psi)[b]
        pr = np.fft.ifftn(box) * ntot          # sum_G c_G exp(+i G.r)
        rho += occ[b] * (pr.real ** 2 + pr.imag ** 2)
    return rho / volume


def g_vectors_sq(lattice, fft) -> tuple[np.ndarray, np.ndarray]:
    """|G|^2 on the FFT grid (index m_d read as m_d - N_d above N_d / 2) and a
    mask that is False at G = 0 and on Nyquist planes."""
    b = reciprocal(lattice)
    ms = []
    keep = np.ones(tuple(fft), dtype=bool)
    for d, n in enumerate(fft):
        m = np.arange(n)
        m = np.where(m > n // 2, m - n, m)
        shape = [1, 1, 1]
        shape[d] = n
        ms.append(m.reshape(shape))
        if n % 2 == 0:
            ny = (np.arange(n) == n // 2).reshape(shape)
            keep &= ~np.broadcast_to(ny, tuple(fft))
    gx = ms[0] * b[0, 0] + ms[1] * b[1, 0] + ms[2] * b[2, 0]
    gy = ms[0] * b[0, 1] + ms[1] * b[1, 1] + ms[2] * b[2, 1]
    gz = ms[0] * b[0, 2] + ms[1] * b[1, 2] + ms[2] * b[2, 2]
    g2 = gx ** 2 + gy ** 2 + gz ** 2
    keep &= g2 > 0
    return g2, keep


def hartree(lattice, rho) -> tuple[np.ndarray, float]:
    """(V_H on the grid, E_H) for the density rho (N1, N2, N3)."""
    fft = rho.shape
    volume = abs(np.linalg.det(np.asarray(lattice, dtype=np.float64)))
    rho_g = np.fft.fftn(rho) / rho.size        # rho(r) = sum_G rho_G exp(i G.r)
    g2, keep = g_vectors_sq(lattice, fft)
    v_g = np.where(keep, 4.0 * np.pi * rho_g / np.where(keep, g2, 1.0), 0.0)
    v_r = (np.fft.ifftn(v_g) * rho.size).real
    e_h = 0.5 * volume * float(np.sum(np.where(keep, 4.0 * np.pi * np.abs(rho_g) ** 2
                                                / np.where(keep, g2, 1.0), 0.0)))
    return v_r, e_h


def lda_xc(rho) -> tuple[np.ndarray, np.ndarray]:
    """(eps_xc, v_xc) per grid point, Slater exchange + Perdew-Zunger correlation."""
    rho = np.asarray(rho, dtype=np.float64)
    ok = rho > RHO_MIN
    r = np.where(ok, rho, 1.0)
    rs = (3.0 / (4.0 * np.pi * r)) ** (1.0 / 3.0)
    ex = -0.75 * (3.0 * r / np.pi) ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex
    p = PZ
    sq = np.sqrt(rs)
    den = 1.0 + p["b1"] * sq + p["b2"] * rs
    ec_hi = p["g"] / den
    vc_hi = ec_hi * (1.0 + 7.0 / 6.0 * p["b1"] * sq + 4.0 / 3.0 * p["b2"] * rs) / den
    lr = np.log(rs)
    ec_lo = p["A"] * lr + p["B"] + p["C"] * rs * lr + p["D"] * rs
    vc_lo = (p["A"] * lr + (p["B"] - p["A"] / 3.0) + 2.0 / 3.0 * p["C"] * rs * lr
             + (2.0 * p["D"] - p["C"]) / 3.0 * rs)
    hi = rs >= 1.0
    exc = np.where(ok, ex + np.where(hi, ec_hi, ec_lo), 0.0)
    vxc = np.where(ok, vx + np.where(hi, vc_hi, vc_lo), 0.0)
    return exc, vxc


def new_potential(lattice, rho, v_ion=None) -> tuple[np.ndarray, dict]:
    """V_LOC = v_ion + V_H + v_xc on the grid, and the energies E_H,
    E_xc = int rho eps_xc dr and int v_xc rho dr."""
    volume = abs(np.linalg.det(np.asarray(lattice, dtype=np.float64)))
    dv = volume / rho.size
    v_h, e_h = hartree(lattice, rho)
    exc, vxc = lda_xc(rho)
    v = v_h + vxc + (0.0 if v_ion is None else v_ion)
    return v, {"e_hartree": e_h, "e_xc": float(np.sum(rho * exc) * dv),
               "int_vxc_rho": float(np.sum(rho * vxc) * dv)}
