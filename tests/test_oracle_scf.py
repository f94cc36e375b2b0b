"""Pins of the oracle's SCF steps (CPU only): density normalisation and
closed forms for one and two plane waves; the Hartree potential of single
Fourier components and of a Gaussian charge against their closed forms, and
the Hartree energy by two routes; the LDA potential as the derivative of the
energy density (central finite differences on both Perdew-Zunger branches),
Slater exchange in its rho form, and the uniform electron gas."""
import numpy as np

from oracle import basis as ob
from oracle import scf
from paper_1709_10010_gb300 import synthetic as syn


def grid_points(lattice, fft):
    f = [np.arange(n) / n for n in fft]
    F = np.stack(np.meshgrid(*f, indexing="ij"), axis=-1)
    return F @ np.asarray(lattice)


def test_density_normalisation_and_single_plane_wave():
    cell = syn.make_cell(1, 8.0, 3, 12.0, 1)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    psi = syn.initial_bands(2, b.npw, 5)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    occ = np.array([2.0, 2.0, 1.5, 0.5, 0.0])
    rho = scf.density(b.miller, b.fft, psi, occ, cell.volume)
    # Parseval: the grid integral of rho is the number of electrons
    assert abs(rho.sum() * cell.volume / rho.size - occ.sum()) < 1e-12
    assert rho.min() >= 0.0
    # one plane wave: a uniform density f / Omega
    one = np.zeros((1, b.npw), complex)
    one[0, 7] = np.exp(0.3j)
    r1 = scf.density(b.miller, b.fft, one, [2.0], cell.volume)
    np.testing.assert_allclose(r1, 2.0 / cell.volume, rtol=1e-13, atol=0)


def test_density_two_plane_waves_closed_form():
    cell = syn.make_cell(2, 7.0, 2, 10.0, 1)
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    i, j = 3, 11
    a, c = 0.6 + 0.2j, -0.3 + 0.7j
    psi = np.zeros((1, b.npw), complex)
    psi[0, i], psi[0, j] = a, c
    rho = scf.density(b.miller, b.fft, psi, [1.0], cell.volume)
    r = grid_points(cell.lattice, b.fft)
    B = ob.reciprocal(cell.lattice)
    gi, gj = b.miller[i] @ B, b.miller[j] @ B
    ph = np.exp(1j * (r @ (gi - gj)))
    ref = (abs(a) ** 2 + abs(c) ** 2 + 2 * np.real(a * np.conj(c) * ph)) / cell.volume
    np.testing.assert_allclose(rho, ref, rtol=0, atol=1e-14)


def test_hartree_of_single_fourier_components():
    lat = np.array([[9.0, 0, 0], [0.4, 8.0, 0], [0.2, -0.3, 10.0]])
    fft = (24, 24, 30)
    r = grid_points(lat, fft)
    B = ob.reciprocal(lat)
    g1 = np.array([1, -2, 1]) @ B
    g2 = np.array([0, 3, -2]) @ B
    rho = 0.05 + 0.02 * np.cos(r @ g1) + 0.01 * np.sin(r @ g2)
    v, e = scf.hartree(lat, rho)
    ref = 4 * np.pi * (0.02 * np.cos(r @ g1) / (g1 @ g1) + 0.01 * np.sin(r @ g2) / (g2 @ g2))
    np.testing.assert_allclose(v, ref, rtol=0, atol=1e-13)
    # E_H by the real-space route: (1/2) int V_H rho
    vol = abs(np.linalg.det(lat))
    assert abs(e - 0.5 * np.sum(v * rho) * vol / rho.size) < 1e-12 * abs(e)
    # closed form: (Omega / 2) 4 pi (|a/2|^2 + |a/2|^2) / g^2 per cosine or sine
    e_ref = 0.5 * vol * 4 * np.pi * (2 * 0.01 ** 2 / (g1 @ g1) + 2 * 0.005 ** 2 / (g2 @ g2))
    assert abs(e - e_ref) < 1e-12 * e_ref


def test_hartree_of_a_gaussian_charge():
    """A periodic Gaussian of charge q and width s: V_H(G) = 4 pi q
    exp(-G^2 s^2 / 2) / (Omega G^2), summed on the grid."""
    a, n, s, q = 10.0, 48, 0.9, 1.7
    lat = np.diag([a, a, a])
    r = grid_points(lat, (n, n, n))
    rho = np.zeros((n, n, n))
    c = np.array([4.0, 5.5, 6.0])
    for sh in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1])).reshape(3, -1).T:
        d = r - c - sh * a
        rho += q * np.exp(-np.sum(d * d, axis=-1) / (2 * s * s)) / (2 * np.pi * s * s) ** 1.5
    v, e = scf.hartree(lat, rho)
    g2, keep = scf.g_vectors_sq(lat, (n, n, n))
    m = np.fft.fftfreq(n, 1.0 / n)
    M = np.stack(np.meshgrid(m, m, m, indexing="ij"), -1)
    G = M * (2 * np.pi / a)
    vg = np.where(keep, 4 * np.pi * q * np.exp(-g2 * s * s / 2) / (a ** 3 * np.where(keep, g2, 1.0)), 0)
    vg = vg * np.exp(-1j * (G @ c))
    ref = (np.fft.ifftn(vg) * n ** 3).real
    np.testing.assert_allclose(v, ref, rtol=0, atol=1e-10)
    assert abs(np.mean(v)) < 1e-12   # neutralising background: V_H has zero mean


def test_lda_potential_is_the_derivative_of_the_energy_density():
    rho = np.array([1e-4, 3e-3, 0.01, 0.2387, 0.24, 0.5, 2.0, 30.0])  # r_s on both sides of 1
    exc, vxc = scf.lda_xc(rho)
    h = 1e-6 * rho
    ep, _ = scf.lda_xc(rho + h)
    em, _ = scf.lda_xc(rho - h)
    fd = ((rho + h) * ep - (rho - h) * em) / (2 * h)
    np.testing.assert_allclose(vxc, fd, rtol=1e-7)


def test_lda_exchange_and_uniform_gas():
    rho = np.array([0.01, 0.1, 1.0])
    rs = (3 / (4 * np.pi * rho)) ** (1 / 3)
    exc, _ = scf.lda_xc(rho)
    ec_lo = 0.0311 * np.log(rs) - 0.048 + 0.0020 * rs * np.log(rs) - 0.0116 * rs
    ec_hi = -0.1423 / (1 + 1.0529 * np.sqrt(rs) + 0.3334 * rs)
    ex = -(3 / (4 * np.pi)) * (9 * np.pi / 4) ** (1 / 3) / rs     # Slater exchange in r_s
    np.testing.assert_allclose(exc, ex + np.where(rs >= 1, ec_hi, ec_lo), rtol=1e-13)
    # zero density: no contribution
    e0, v0 = scf.lda_xc(np.array([0.0, 1e-30]))
    assert np.all(e0 == 0) and np.all(v0 == 0)
    # uniform gas: E_xc = Omega rho eps_xc, and V_H = 0
    lat = np.diag([6.0, 6.0, 6.0])
    v, en = scf.new_potential(lat, np.full((12, 12, 12), 0.1))
    assert abs(en["e_hartree"]) < 1e-15
    assert abs(en["e_xc"] - 216.0 * 0.1 * scf.lda_xc(np.array([0.1]))[0][0]) < 1e-12
