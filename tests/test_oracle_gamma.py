"""Pins of the oracle's Gamma-point pieces (CPU only): the half sphere covers the
sphere exactly once with its mirror; expanded coefficients are real functions
on the grid; H keeps real functions real (conjugate symmetry of the result);
the two-bands-per-FFT identity against band-by-band local terms; the free
electron case; a closed form for a single cosine band."""
import numpy as np

from oracle import basis as ob
from oracle import gamma as og
from oracle import hamiltonian as oh
from paper_1709_10010_gb300 import synthetic as syn


def gamma_case(seed=0, a=8.0, natoms=3, ecut_ry=12.0, lmax=2):
    cell = syn.make_cell(seed, a, natoms, ecut_ry, lmax)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    return cell, b, syn.potential_grid(cell, b.fft), syn.projectors(cell, b.miller), syn.d_diagonal(cell)


def test_half_sphere_partition():
    cell, b, v, beta, D = gamma_case()
    half, neg = og.half_sphere(b.miller)
    assert len(half) == (b.npw + 1) // 2
    both = np.concatenate([half, neg])
    # every plane wave appears, G = 0 twice (it is its own mirror), nothing else repeats
    counts = np.bincount(both, minlength=b.npw)
    g0 = np.nonzero(np.all(b.miller == 0, axis=1))[0][0]
    assert counts[g0] == 2 and np.all(np.delete(counts, g0) == 1)
    np.testing.assert_array_equal(b.miller[neg], -b.miller[half])
    assert np.all(np.diff(half) > 0)   # public order kept


def test_expanded_bands_are_real_functions():
    cell, b, v, beta, D = gamma_case(1)
    half, _ = og.half_sphere(b.miller)
    psi = syn.initial_bands(3, len(half), 4)
    full = og.expand(b.miller, psi)
    n1, n2, n3 = b.fft
    for k in range(4):
        box = np.zeros(b.fft, complex)
        box[b.miller[:, 0] % n1, b.miller[:, 1] % n2, b.miller[:, 2] % n3] = full[k]
        r = np.fft.ifftn(box)
        assert np.abs(r.imag).max() <= 1e-15 * np.abs(r.real).max() + 1e-300


def test_h_keeps_real_functions_real():
    cell, b, v, beta, D = gamma_case(2)
    half, neg = og.half_sphere(b.miller)
    full = og.expand(b.miller, syn.initial_bands(4, len(half), 3))
    h = oh.apply_h(b, v, beta, D, full)
    np.testing.assert_allclose(h[:, neg], np.conj(h[:, half]), rtol=0, atol=1e-12 * np.abs(h).max())


def test_two_bands_per_fft_identity():
    cell, b, v, beta, D = gamma_case(3)
    half, _ = og.half_sphere(b.miller)
    psi = syn.initial_bands(5, len(half), 2)
    two = og.local_two_bands(b, v, psi)
    one = oh.local_fft(b.miller, b.fft, v, og.expand(b.miller, psi))[:, half]
    np.testing.assert_allclose(two, one, rtol=0, atol=1e-13 * np.abs(one).max())


def test_free_electrons_and_a_cosine_band():
    cell, b, v, beta, D = gamma_case(4)
    half, _ = og.half_sphere(b.miller)
    psi = syn.initial_bands(6, len(half), 2)
    out = og.apply_h_gamma(b, np.zeros(b.fft), None, None, psi)
    kin = b.kinetic[half]
    psi0 = psi.copy()
    psi0[:, 0] = psi0[:, 0].real            # c(0) is real for a real function
    np.testing.assert_allclose(out, kin[None, :] * psi0, rtol=0, atol=1e-13)
    # a single cosine cos(G.r) (c(G) = c(-G) = 1/2) in the constant potential V = c
    one = np.zeros((1, len(half)), complex)
    one[0, 5] = 0.5
    out = og.apply_h_gamma(b, np.full(b.fft, 0.3), None, None, one)
    ref = np.zeros_like(one)
    ref[0, 5] = 0.5 * (kin[5] + 0.3)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-14)
