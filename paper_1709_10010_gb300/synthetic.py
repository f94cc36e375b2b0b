"""Seeded synthetic inputs for the plane-wave Hamiltonian: cells, local potential,
projectors, nonlocal coefficients and starting bands.

This module only *synthesises inputs*; it holds none of the arithmetic of the
Hamiltonian application or of the eigensolver.  Both the CPU oracle (under
``oracle/``) and the CUDA library consume what it produces, so the two sides
always see bit-identical inputs.

Every random draw comes from ``numpy.random.default_rng`` (PCG64) seeded as
documented per function, so a (config, seed) pair fixes every array.

Physical model of the inputs (Hartree atomic units, bohr):

* local potential: a periodic sum of attractive Gaussians per atom,
  ``V_I(r) = A_I exp(-|r-R_I|^2 / (2 w_I^2))`` with ``A_I ~ U(-2,-0.5)`` Ha and
  ``w_I ~ U(0.8,1.5)`` bohr.  Its Fourier coefficients are
  ``V(G) = sum_I A_I (2 pi)^{3/2} w_I^3 / Omega  exp(-G^2 w_I^2/2) exp(-i G.R_I)``,
  truncated to ``|G| <= 2 G_c`` (the density cutoff of the plane-wave method,
  Sec. "Advanced implementation of exact (Fock) exchange": ``G_max = 2 G_c``),
  and sampled on the real-space FFT grid.
* projectors (the ``beta`` of Eq. pauli_ks, Sec. "Fully relativistic projector
  augmented-wave method"): Gaussian radial functions ``r^l exp(-r^2/(2 rc^2))``
  with ``rc = 1`` bohr times real spherical harmonics, whose plane-wave
  coefficients at ``q = k+G`` are
  ``(4 pi/sqrt(Omega)) (-i)^l sqrt(pi/2) rc^{2l+3} exp(-q^2 rc^2/2) S_lm(q) exp(-i q.R_I)``
  with ``S_lm(q) = |q|^l Y_lm(q_hat)`` the real solid harmonics.
* ``D``: diagonal, one ``U(-1,1)`` Ha value per (atom, l), shared over m.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Projectors per atom for l_max = 1 (s+p) and l_max = 2 (s,p,d).
PROJ_PER_ATOM = {0: 1, 1: 4, 2: 9}


@dataclasses.dataclass
class Cell:
    lattice: np.ndarray      # (3,3) rows a1, a2, a3 in bohr
    kpoint: np.ndarray       # (3,) fractional, in units of the reciprocal vectors b_i
    ecut_ha: float           # wavefunction cutoff in Hartree: 1/2 |k+G|^2 <= ecut_ha
    positions: np.ndarray    # (natoms, 3) cartesian bohr
    amp: np.ndarray          # (natoms,) Gaussian depth A_I in Ha
    width: np.ndarray        # (natoms,) Gaussian width w_I in bohr
    lmax: int                # projector channels l = 0..lmax
    d_l: np.ndarray          # (natoms, lmax+1) D value per (atom, l) in Ha
    rc: float = 1.0          # projector Gaussian radius in bohr

    @property
    def natoms(self) -> int:
        return int(self.positions.shape[0])

    @property
    def nproj(self) -> int:
        return self.natoms * PROJ_PER_ATOM[self.lmax]

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))

    def desc(self) -> dict:
        """Arguments for creating a system with this cell."""
        return dict(lattice=self.lattice.copy(), kpoint=self.kpoint.copy(),
                    ecut_ha=self.ecut_ha)


def make_cell(seed: int, a, natoms: int, ecut_ry: float, lmax: int,
              kpoint=(0.0, 0.0, 0.0)) -> Cell:
    """A cell with uniformly random atoms.

    ``a`` is a cubic edge (float) or a (3,3) lattice.  Draw order from
    ``default_rng(seed)``: fractional positions (natoms,3) ~ U[0,1), depths,
    widths, then the D values (natoms, lmax+1) ~ U(-1,1).
    """
    lattice = (np.diag([float(a)] * 3) if np.ndim(a) == 0
               else np.asarray(a, dtype=np.float64).reshape(3, 3))
    rng = np.random.default_rng(seed)
    frac = rng.uniform(0.0, 1.0, size=(natoms, 3))
    amp = rng.uniform(-2.0, -0.5, size=natoms)
    width = rng.uniform(0.8, 1.5, size=natoms)
    d_l = rng.uniform(-1.0, 1.0, size=(natoms, lmax + 1))
    return Cell(lattice=lattice, kpoint=np.asarray(kpoint, dtype=np.float64),
                ecut_ha=0.5 * float(ecut_ry), positions=frac @ lattice, amp=amp,
                width=width, lmax=int(lmax), d_l=d_l)


def reciprocal_vectors(lattice: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def potential_grid(cell: Cell, fft) -> np.ndarray:
    """V_loc(r) on the N1 x N2 x N3 grid, C order (i3 fastest), float64.

    Grid point (i1,i2,i3) is r = sum_d (i_d/N_d) a_d.  The Gaussian Fourier
    series is truncated to |G| <= 2 G_c with G_c = sqrt(2 ecut) and summed on the
    grid with numpy's inverse FFT (input synthesis only).
    """
    n1, n2, n3 = (int(x) for x in fft)
    bvec = reciprocal_vectors(cell.lattice)
    m = [np.fft.fftfreq(n, 1.0 / n).astype(np.int64) for n in (n1, n2, n3)]
    M1, M2, M3 = np.meshgrid(m[0], m[1], m[2], indexing="ij")
    gx = M1 * bvec[0, 0] + M2 * bvec[1, 0] + M3 * bvec[2, 0]
    gy = M1 * bvec[0, 1] + M2 * bvec[1, 1] + M3 * bvec[2, 1]
    gz = M1 * bvec[0, 2] + M2 * bvec[1, 2] + M3 * bvec[2, 2]
    g2 = gx * gx + gy * gy + gz * gz
    gmax2 = 4.0 * 2.0 * cell.ecut_ha          # (2 G_c)^2
    mask = g2 <= gmax2
    frac = cell.positions @ np.linalg.inv(cell.lattice)
    vg = np.zeros((n1, n2, n3), dtype=np.complex128)
    omega = cell.volume
    for i in range(cell.natoms):
        ph = [np.exp(-2j * np.pi * m[d] * frac[i, d]) for d in range(3)]
        phase = ph[0][:, None, None] * ph[1][None, :, None] * ph[2][None, None, :]
        w = cell.width[i]
        pref = cell.amp[i] * (2.0 * np.pi) ** 1.5 * w ** 3 / omega
        vg += pref * np.exp(-0.5 * g2 * w * w) * phase
    vg[~mask] = 0.0
    vr = np.fft.ifftn(vg) * (n1 * n2 * n3)
    return np.ascontiguousarray(vr.real)


def _real_solid_harmonics(qx, qy, qz, lmax):
    """S_lm(q) = |q|^l Y_lm(q_hat) for l <= lmax, standard real harmonics.

    Order per l: l=0: [1]; l=1: [y, z, x]; l=2: [xy, yz, 3z^2-r^2, xz, x^2-y^2].
    """
    out = [np.full_like(qx, 0.5 / math.sqrt(math.pi))]
    if lmax >= 1:
        c1 = math.sqrt(3.0 / (4.0 * math.pi))
        out += [c1 * qy, c1 * qz, c1 * qx]
    if lmax >= 2:
        c2 = math.sqrt(15.0 / (4.0 * math.pi))
        c20 = math.sqrt(5.0 / (16.0 * math.pi))
        c22 = math.sqrt(15.0 / (16.0 * math.pi))
        q2 = qx * qx + qy * qy + qz * qz
        out += [c2 * qx * qy, c2 * qy * qz, c20 * (3.0 * qz * qz - q2),
                c2 * qx * qz, c22 * (qx * qx - qy * qy)]
    return out


def projector_l_of_column(cell: Cell) -> np.ndarray:
    """Angular momentum l of each projector column (atom-major, then l, then m)."""
    ls = []
    for _ in range(cell.natoms):
        for l in range(cell.lmax + 1):
            ls += [l] * (2 * l + 1)
    return np.asarray(ls, dtype=np.int64)


def projectors(cell: Cell, miller: np.ndarray) -> np.ndarray:
    """beta as a (P, npw) complex128 array: row j is projector j sampled at the
    plane waves ``miller`` (npw, 3) in the order given.  Row-major (P, npw) is the
    same memory as column-major npw x P.  Column order: atom, then l, then m."""
    miller = np.asarray(miller, dtype=np.int64)
    bvec = reciprocal_vectors(cell.lattice)
    f = miller.astype(np.float64) + cell.kpoint[None, :]
    qx = f[:, 0] * bvec[0, 0] + f[:, 1] * bvec[1, 0] + f[:, 2] * bvec[2, 0]
    qy = f[:, 0] * bvec[0, 1] + f[:, 1] * bvec[1, 1] + f[:, 2] * bvec[2, 1]
    qz = f[:, 0] * bvec[0, 2] + f[:, 1] * bvec[1, 2] + f[:, 2] * bvec[2, 2]
    q2 = qx * qx + qy * qy + qz * qz
    rc = cell.rc
    harm = _real_solid_harmonics(qx, qy, qz, cell.lmax)
    pref = 4.0 * np.pi / math.sqrt(cell.volume)
    rows = []
    for i in range(cell.natoms):
        R = cell.positions[i]
        sf = np.exp(-1j * (qx * R[0] + qy * R[1] + qz * R[2]))
        k = 0
        for l in range(cell.lmax + 1):
            radial = math.sqrt(math.pi / 2.0) * rc ** (2 * l + 3) * np.exp(-0.5 * q2 * rc * rc)
            for _m in range(2 * l + 1):
                rows.append(pref * (-1j) ** l * radial * harm[k] * sf)
                k += 1
    if not rows:
        return np.zeros((0, miller.shape[0]), dtype=np.complex128)
    return np.ascontiguousarray(np.stack(rows))


def d_diagonal(cell: Cell) -> np.ndarray:
    """Diagonal of D, one value per projector column (shared over m)."""
    out = []
    for i in range(cell.natoms):
        for l in range(cell.lmax + 1):
            out += [cell.d_l[i, l]] * (2 * l + 1)
    return np.asarray(out, dtype=np.float64)


def initial_bands(seed: int, npw: int, nb: int) -> np.ndarray:
    """Starting bands, (nb, npw) complex128 (row = band, i.e. column-major npw x nb).
    Real and imaginary parts ~ N(0,1) from ``default_rng([seed, 1])``."""
    rng = np.random.default_rng([int(seed), 1])
    re = rng.standard_normal((nb, npw))
    im = rng.standard_normal((nb, npw))
    return re + 1j * im


def random_hermitian(seed: int, n: int) -> np.ndarray:
    """A random complex Hermitian n x n matrix, entries ~ N(0,1) (test input)."""
    rng = np.random.default_rng([int(seed), 2])
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (a + a.conj().T)


# Workloads with the shapes of the plane-wave systems the method targets.
CONFIGS = {
    # a=10 bohr, 20 Ry, 8 atoms, s+p projectors, 16 bands: Npw 1503, grid 30^3
    "small": dict(a=10.0, natoms=8, ecut_ry=20.0, lmax=1, nb=16),
    # a=20 bohr, 40 Ry, 64 atoms, s,p,d projectors, 128 bands: Npw 34265, grid 90^3
    "medium": dict(a=20.0, natoms=64, ecut_ry=40.0, lmax=2, nb=128),
    # a=30 bohr, 50 Ry, 216 atoms, s,p,d projectors, 512 bands: Npw 161235, grid 144^3
    "large": dict(a=30.0, natoms=216, ecut_ry=50.0, lmax=2, nb=512),
}


def config_cell(name: str, seed: int = 0) -> Cell:
    c = CONFIGS[name]
    return make_cell(seed, c["a"], c["natoms"], c["ecut_ry"], c["lmax"])


# 2x2x2 Monkhorst-Pack grid (fractional): all eight (+-1/4, +-1/4, +-1/4)
MP222 = [(sx * 0.25, sy * 0.25, sz * 0.25) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]


def batched_workload(ncells: int = 32, seed: int = 0, ecut_ry: float = 30.0):
    """Independent systems of the batched workload: ``ncells`` cubic cells with
    edge ~ U(8, 14) bohr and 4-16 atoms (s,p,d projectors), 30 Ry, each at the
    eight k-points of a 2x2x2 Monkhorst-Pack grid, 24-48 bands per cell.
    Draws from ``default_rng([seed, 4])``: per cell edge, atom count, band count.
    Returns a list of (cell, nb), cells at a k-point sharing the cell's atoms."""
    rng = np.random.default_rng([int(seed), 4])
    out = []
    for c in range(ncells):
        a = float(rng.uniform(8.0, 14.0))
        natoms = int(rng.integers(4, 17))
        nb = int(rng.integers(24, 49))
        for k in MP222:
            out.append((make_cell(10_000 + 100 * seed + c, a, natoms, ecut_ry, 2, kpoint=k), nb))
    return out
