"""Plane-wave basis of the oracle (TEST INFRASTRUCTURE; see ``oracle/__init__``).

* The basis is the sphere ``{G : 1/2 |k+G|^2 <= ecut}`` (plane-wave coefficients
  c_{k,n}(G) of the Kohn-Sham orbitals, Sec. "New parallelization levels"), with
  membership decided in FP64 from the integer Miller indices, inclusive with a
  relative slack of 1e-12 so that plane waves lying exactly on the cutoff are
  kept whatever the last-bit rounding of |k+G|^2.
* Ordering (Sec. "Large-record data file format" asks for a reproducible,
  machine-independent ordering including inside shells of equal modulus):
  ascending |k+G|^2; plane waves whose |k+G|^2 agree to a relative 1e-10 form one
  shell and are ordered lexicographically by signed (m1, m2, m3).
* FFT box: the product psi*V needs G up to 2 G_c (Sec. "Advanced implementation
  of exact (Fock) exchange": G_max = 2 G_c, E = 4 E_c), so a convolution free of
  aliasing on the sphere needs N_i >= 4 mmax_i + 1; N_i is the smallest even
  2,3,5-smooth integer at or above that.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def reciprocal(lattice) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def kplusg_sq(lattice, kpoint, miller) -> np.ndarray:
    """|k+G|^2 in FP64 for integer Miller rows: q = sum_i (m_i + k_i) b_i, each
    cartesian component summed in the order i = 1, 2, 3, then qx^2+qy^2+qz^2."""
    b = reciprocal(lattice)
    f = np.asarray(miller, dtype=np.float64) + np.asarray(kpoint, dtype=np.float64)[None, :]
    qx = f[:, 0] * b[0, 0] + f[:, 1] * b[1, 0] + f[:, 2] * b[2, 0]
    qy = f[:, 0] * b[0, 1] + f[:, 1] * b[1, 1] + f[:, 2] * b[2, 1]
    qz = f[:, 0] * b[0, 2] + f[:, 1] * b[1, 2] + f[:, 2] * b[2, 2]
    return qx * qx + qy * qy + qz * qz


def smooth_even_at_least(n: int) -> int:
    """Smallest even integer >= n whose prime factors are all in {2, 3, 5}."""
    m = max(int(n), 2)
    while True:
        if m % 2 == 0:
            r = m
            for p in (2, 3, 5):
                while r % p == 0:
                    r //= p
            if r == 1:
                return m
        m += 1


@dataclasses.dataclass
class Basis:
    miller: np.ndarray   # (npw, 3) int64, public order
    q2: np.ndarray       # (npw,) |k+G|^2
    kinetic: np.ndarray  # (npw,) 1/2 |k+G|^2 (Hartree)
    shell: np.ndarray    # (npw,) shell id (0-based, ascending |k+G|^2)
    fft: tuple           # (N1, N2, N3)

    @property
    def npw(self) -> int:
        return int(self.miller.shape[0])


def sphere(lattice, kpoint, ecut_ha, fft=None) -> Basis:
    """The plane-wave sphere in public order; ``fft`` overrides the box size."""
    lattice = np.asarray(lattice, dtype=np.float64)
    kpoint = np.asarray(kpoint, dtype=np.float64)
    gc = np.sqrt(2.0 * ecut_ha)
    # |m_i + k_i| = |q . a_i| / (2 pi) <= G_c |a_i| / (2 pi)
    bound = [int(np.floor(gc * np.linalg.norm(lattice[i]) / (2.0 * np.pi) + abs(kpoint[i]))) + 1
             for i in range(3)]
    r = [np.arange(-bound[i], bound[i] + 1) for i in range(3)]
    M1, M2, M3 = np.meshgrid(r[0], r[1], r[2], indexing="ij")
    cand = np.stack([M1.ravel(), M2.ravel(), M3.ravel()], axis=1)
    q2 = kplusg_sq(lattice, kpoint, cand)
    keep = 0.5 * q2 <= ecut_ha * (1.0 + 1e-12)   # inclusive, robust to 1-ulp rounding
    cand, q2 = cand[keep], q2[keep]
    # sort by |k+G|^2, cut into shells, then lexicographic inside each shell
    o = np.lexsort((cand[:, 2], cand[:, 1], cand[:, 0], q2))
    cand, q2 = cand[o], q2[o]
    new_shell = np.zeros(q2.shape[0], dtype=bool)
    if q2.shape[0]:
        new_shell[0] = True
        new_shell[1:] = (q2[1:] - q2[:-1]) > 1e-10 * q2[1:]
    shell = np.cumsum(new_shell) - 1
    o = np.lexsort((cand[:, 2], cand[:, 1], cand[:, 0], shell))
    cand, q2, shell = cand[o], q2[o], shell[o]
    mmax = np.abs(cand).max(axis=0) if cand.shape[0] else np.zeros(3, dtype=np.int64)
    if fft is None:
        fft = tuple(smooth_even_at_least(4 * int(mmax[i]) + 1) for i in range(3))
    fft = tuple(int(x) for x in fft)
    return Basis(miller=cand.astype(np.int64), q2=q2, kinetic=0.5 * q2,
                 shell=shell.astype(np.int64), fft=fft)
