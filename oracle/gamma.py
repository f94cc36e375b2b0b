"""Real wavefunctions at the Gamma point (TEST INFRASTRUCTURE; see
``oracle/__init__``).

At k = 0 a real psi(r) has c(-G) = conj(c(G)), so half of the sphere carries
all its information (the Gamma-only storage of Sec. "Advanced implementation
of exact (Fock) exchange", ACE paragraph, and of the real-wavefunction codes of
Sec. "Many-body perturbation theory").  The half sphere: G = 0 and every G
whose first nonzero Miller index is positive, in the public order; c(0) is
real.

* ``apply_h_gamma`` is the plain definition: expand to the full sphere, apply
  H (``hamiltonian.apply_h``), keep the half.  H maps real functions to real
  functions when V(r) is real and the projectors satisfy beta(-G) =
  conj(beta(G)) (true of the generated projectors at k = 0) with D real.
* ``local_two_bands`` is the route of the GPU path written out independently:
  two real bands share one complex FFT, Psi = psi_1 + i psi_2, and
  (V psi_1)(G) = (Phi(G) + conj(Phi(-G)))/2, (V psi_2)(G) = (Phi(G) -
  conj(Phi(-G)))/(2i) with Phi the transform of V Psi.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as oh


def half_sphere(miller) -> tuple[np.ndarray, np.ndarray]:
    """(indices of the half sphere in the public order, index of -G for each)."""
    m = np.asarray(miller)
    pos = (m[:, 0] > 0) | ((m[:, 0] == 0) & (m[:, 1] > 0)) | \
          ((m[:, 0] == 0) & (m[:, 1] == 0) & (m[:, 2] >= 0))
    half = np.nonzero(pos)[0]
    where = {tuple(r): i for i, r in enumerate(m.tolist())}
    neg = np.array([where[tuple((-m[i]).tolist())] for i in half])
    return half, neg


def expand(miller, psi_half) -> np.ndarray:
    """Full-sphere coefficients (nb, npw) of real functions given on the half
    sphere (nb, npw_half); the imaginary part of c(0) is dropped."""
    half, neg = half_sphere(miller)
    psi_half = np.atleast_2d(psi_half)
    out = np.zeros((psi_half.shape[0], len(miller)), dtype=np.complex128)
    out[:, neg] = np.conj(psi_half)
    out[:, half] = psi_half
    g0 = np.nonzero(np.all(np.asarray(miller) == 0, axis=1))[0]
    out[:, g0] = out[:, g0].real
    return out


def apply_h_gamma(basis, v_r, beta, D, psi_half) -> np.ndarray:
    """H applied to real bands given on the half sphere, returned on the half."""
    half, _ = half_sphere(basis.miller)
    return oh.apply_h(basis, v_r, beta, D, expand(basis.miller, psi_half))[:, half]


def local_two_bands(basis, v_r, psi_half) -> np.ndarray:
    """The local term of two real bands (2, npw_half) through one complex FFT."""
    half, neg = half_sphere(basis.miller)
    full = expand(basis.miller, psi_half)
    Psi = full[0] + 1j * full[1]
    Phi = oh.local_fft(basis.miller, basis.fft, v_r, Psi[None, :])[0]
    p, q = Phi[half], np.conj(Phi[neg])
    return np.stack([(p + q) / 2, (p - q) / 2j])
