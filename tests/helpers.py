"""Shared test set-up: seeded inputs from the generator plus the oracle's basis.
(Test infrastructure; imports the oracle.)"""
import numpy as np

from oracle import basis as ob
from paper_1709_10010_gb300 import synthetic as syn


def case(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1, k=(0, 0, 0)):
    """A cell, its oracle basis, V(r), beta (public order) and diagonal D."""
    cell = syn.make_cell(seed, a, natoms, ecut_ry, lmax, kpoint=k)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    return cell, b, v, beta, D


def rel_err(x, ref):
    """max |x - ref| / max |ref| over all entries."""
    return float(np.abs(np.asarray(x) - np.asarray(ref)).max() / np.abs(np.asarray(ref)).max())
