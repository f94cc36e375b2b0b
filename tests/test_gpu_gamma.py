"""Real bands at k = 0 on the GPU (two real bands per complex FFT, half-sphere
storage) against the oracle's plain definition: expand the half sphere with
c(-G) = conj c(G), apply the FP64 H, keep the half.  Element by element, FP64
bar 1e-12 and mixed bar 1e-4 of max |H psi| (the bars of the complex apply:
packing and unpacking are exact up to one FP64 halving)."""
import numpy as np
import pytest

from oracle import gamma as og
from oracle import hamiltonian as oh
from paper_1709_10010_gb300 import synthetic as syn
from tests.helpers import case, rel_err

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def torch():
    import torch
    from paper_1709_10010_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


def make_system(cell, v, beta, D, precision="fp64"):
    import paper_1709_10010_gb300 as pwh
    s = pwh.System.from_cell(cell, precision=precision)
    s.set_potential(v)
    if beta is not None:
        s.set_projectors(beta, D)
    return s


def real_bands(seed, nh, nb, b):
    """Half-sphere bands of real functions (c(0) real)."""
    psi = syn.initial_bands(seed, nh, nb)
    half, _ = og.half_sphere(b.miller)
    g0 = int(np.nonzero(np.all(b.miller[half] == 0, axis=1))[0][0])
    psi[:, g0] = psi[:, g0].real
    return psi


CASES = [
    dict(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1),
    dict(seed=1, a=10.0, natoms=8, ecut_ry=20.0, lmax=1),   # the 1503-plane-wave cell
    dict(seed=4, a=9.0, natoms=3, ecut_ry=16.0, lmax=2),
]


@pytest.mark.parametrize("kw", CASES)
def test_half_sphere_matches_oracle(torch, kw):
    cell, b, v, beta, D = case(**kw)
    s = make_system(cell, v, beta, D)
    half, _ = og.half_sphere(b.miller)
    np.testing.assert_array_equal(s.gamma_half(), half)
    assert len(half) == (b.npw + 1) // 2


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("nb", [1, 2, 7, 40])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_apply_h_gamma_parity(torch, kw, nb, mode):
    cell, b, v, beta, D = case(**kw)
    s = make_system(cell, v, beta, D, mode)
    half, _ = og.half_sphere(b.miller)
    psi = real_bands(20 + nb, len(half), nb, b)
    ref = og.apply_h_gamma(b, v, beta, D, psi)
    out = s.apply_h_gamma(torch.from_numpy(psi).cuda()).cpu().numpy()
    s.sync()
    assert rel_err(out, ref) <= (FP64_TOL if mode == "fp64" else MIXED_TOL)


def test_gamma_matches_complex_apply(torch):
    """The half of the complex apply of the expanded bands (same library, other
    route): FP64 results agree to rounding."""
    cell, b, v, beta, D = case(seed=1, a=10.0, natoms=8, ecut_ry=20.0, lmax=1)
    s = make_system(cell, v, beta, D)
    half, _ = og.half_sphere(b.miller)
    psi = real_bands(3, len(half), 9, b)
    full = s.apply_h(torch.from_numpy(og.expand(b.miller, psi)).cuda()).cpu().numpy()[:, half]
    out = s.apply_h_gamma(torch.from_numpy(psi).cuda()).cpu().numpy()
    assert rel_err(out, full) <= 1e-13


def test_gamma_strided_full_real_D_and_no_projectors(torch):
    cell, b, v, beta, D = case(seed=5, a=8.0, natoms=3, ecut_ry=14.0, lmax=2)
    rng = np.random.default_rng(1)
    P = beta.shape[0]
    Df = rng.standard_normal((P, P))
    Df = 0.5 * (Df + Df.T) + 0j
    s = make_system(cell, v, beta, Df)
    half, _ = og.half_sphere(b.miller)
    nh = len(half)
    psi = real_bands(7, nh, 5, b)
    # bands as rows of a wider tensor (ld > npw_half), result into a strided view
    big = torch.zeros((5, nh + 37), dtype=torch.complex128, device="cuda")
    big[:, :nh] = torch.from_numpy(psi).cuda()
    hbig = torch.zeros((5, nh + 11), dtype=torch.complex128, device="cuda")
    s.apply_h_gamma(big[:, :nh], hbig[:, :nh])
    ref = og.apply_h_gamma(b, v, beta, Df, psi)
    assert rel_err(hbig[:, :nh].cpu().numpy(), ref) <= FP64_TOL
    assert float(hbig[:, nh:].abs().max()) == 0.0       # nothing written past npw_half
    # no projectors: kinetic + local only
    s2 = make_system(cell, v, None, None)
    ref2 = og.apply_h_gamma(b, v, None, None, psi)
    assert rel_err(s2.apply_h_gamma(torch.from_numpy(psi).cuda()).cpu().numpy(), ref2) <= FP64_TOL


def test_gamma_rejects_what_breaks_reality(torch):
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(seed=6, a=8.0, natoms=2, ecut_ry=12.0, lmax=1)
    half, _ = og.half_sphere(b.miller)
    psi = torch.from_numpy(real_bands(1, len(half), 2, b)).cuda()
    # projectors with a random phase per plane wave: beta(-G) != conj beta(G)
    rng = np.random.default_rng(2)
    bad = beta * np.exp(1j * rng.uniform(0, 2 * np.pi, b.npw))[None, :]
    s = make_system(cell, v, bad, D)
    with pytest.raises(pwh.PwhError) as e:
        s.apply_h_gamma(psi)
    assert e.value.status == 1
    # a full D with imaginary parts
    P = beta.shape[0]
    Dc = np.diag(D).astype(complex)
    Dc[0, 1], Dc[1, 0] = 0.3j, -0.3j
    s = make_system(cell, v, beta, Dc)
    with pytest.raises(pwh.PwhError) as e:
        s.apply_h_gamma(psi)
    assert e.value.status == 1
    # setting valid projectors again clears the verdict
    s.set_projectors(beta, D)
    s.apply_h_gamma(psi)
    s.sync()
    # k != 0
    cellk, bk, vk, betak, Dk = case(seed=6, a=8.0, natoms=2, ecut_ry=12.0, lmax=1, k=(0.25, 0, 0))
    sk = make_system(cellk, vk, betak, Dk)
    with pytest.raises(pwh.PwhError) as e:
        sk.gamma_half()
    assert e.value.status == 1


def test_gamma_medium_cell(torch):
    """The 34,265-plane-wave cell (90^3 box, 576 projectors), both precisions,
    on 16 real bands (8 complex FFTs), every element."""
    cell = syn.config_cell("medium", 0)
    from oracle import basis as ob
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    half, _ = og.half_sphere(b.miller)
    psi = real_bands(9, len(half), 16, b)
    ref = og.apply_h_gamma(b, v, beta, D, psi)
    for mode, tol in (("fp64", FP64_TOL), ("mixed", MIXED_TOL)):
        s = make_system(cell, v, beta, D, mode)
        out = s.apply_h_gamma(torch.from_numpy(psi).cuda()).cpu().numpy()
        s.sync()
        assert rel_err(out, ref) <= tol, (mode, rel_err(out, ref))
        s.close()


# ------------------------------------------------------- real-band eigensolver
def full_norms(b, R_half):
    """Norms over the full sphere of real bands given on the half sphere."""
    return np.linalg.norm(og.expand(b.miller, R_half), axis=1)


@pytest.mark.parametrize("kw,nb", [
    (dict(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1), 8),
    (dict(seed=1, a=10.0, natoms=8, ecut_ry=20.0, lmax=1), 16),   # the 1503-plane-wave cell
    (dict(seed=4, a=9.0, natoms=3, ecut_ry=16.0, lmax=2), 11),
])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_davidson_gamma_matches_dense_eigh(torch, kw, nb, mode):
    """Lowest eigenpairs of real bands against LAPACK on the oracle's dense H
    (the complex H at k = 0 has the same spectrum); eigenvectors as real
    functions: orthonormal over the full sphere, residual by the oracle's H."""
    cell, b, v, beta, D = case(**kw)
    s = make_system(cell, v, beta, D, mode)
    half, _ = og.half_sphere(b.miller)
    psi = torch.from_numpy(real_bands(5, len(half), nb, b)).cuda()
    mixed = mode == "mixed"
    eig, st, status = s.davidson_gamma(psi, tol=1e-9, mixed=mixed, switch_tol=1e-3,
                                       jd_inner=20 if mixed else 0)
    assert status == 0 and st["max_resid"] <= 1e-9
    ref = np.linalg.eigvalsh(oh.dense_h(b, v, beta, D))[:nb]
    assert np.abs(eig - ref).max() <= (1e-10 if mode == "fp64" else 1e-8), np.abs(eig - ref).max()
    X = psi.cpu().numpy()
    g0 = int(np.nonzero(np.all(b.miller[half] == 0, axis=1))[0][0])
    assert np.abs(X[:, g0].imag).max() == 0.0                  # c(0) real on output
    F = og.expand(b.miller, X)
    assert np.abs(F.conj() @ F.T - np.eye(nb)).max() < 1e-12
    R = og.apply_h_gamma(b, v, beta, D, X) - eig[:, None] * X
    assert full_norms(b, R).max() <= 2e-9


def test_davidson_gamma_medium_vs_complex(torch):
    """The 34,265-plane-wave cell, 128 real bands (mixed + Jacobi-Davidson)
    against the complex solver on the same system: eigenvalues within 1e-8 Ha;
    sampled eigenvectors' residuals by the oracle's H."""
    cell = syn.config_cell("medium", 0)
    from oracle import basis as ob
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    beta = syn.projectors(cell, b.miller)
    D = syn.d_diagonal(cell)
    s = make_system(cell, v, beta, D, "mixed")
    nb = 128
    half, _ = og.half_sphere(b.miller)
    psig = torch.from_numpy(real_bands(0, len(half), nb, b)).cuda()
    eg, stg, status = s.davidson_gamma(psig, tol=1e-8, mixed=True, switch_tol=1e-3, jd_inner=20)
    assert status == 0 and stg["max_resid"] <= 1e-8
    psic = torch.from_numpy(syn.initial_bands(0, b.npw, nb)).cuda()
    ec, stc, status = s.davidson(psic, tol=1e-8, mixed=True, switch_tol=1e-3, jd_inner=20)
    assert status == 0
    assert np.abs(eg - ec).max() <= 1e-8, np.abs(eg - ec).max()
    X = psig.cpu().numpy()
    pick = [0, 1, 63, 126, 127]
    R = og.apply_h_gamma(b, v, beta, D, X[pick]) - eg[pick, None] * X[pick]
    assert full_norms(b, R).max() <= 2e-8
    s.close()


def test_davidson_gamma_rejects_k_shift(torch):
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(seed=2, a=9.0, natoms=3, ecut_ry=12.0, lmax=2, k=(0.25, 0, 0))
    s = make_system(cell, v, beta, D)
    psi = torch.zeros((4, (b.npw + 1) // 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(pwh.PwhError) as e:
        s.davidson_gamma(psi)
    assert e.value.status == 1
