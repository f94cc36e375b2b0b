"""The SCF steps on the GPU (pwh_density, pwh_hartree_xc) against the oracle
(oracle/scf.py) through the C ABI, element by element: cubic, k-shifted and
general cells, compiled and runtime-plan box sizes, occupations with zeros,
and the 34,265-plane-wave cell at its 90^3 box.  Bar: 1e-12 of the largest
value (FP64 on both sides; the FFT routes differ only in rounding order)."""
import numpy as np
import pytest

from oracle import scf as oscf
from paper_1709_10010_gb300 import synthetic as syn
from tests.helpers import case, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    from paper_1709_10010_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


CASES = [
    dict(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1),
    dict(seed=2, a=9.0, natoms=3, ecut_ry=16.0, lmax=2, k=(0.25, -0.25, 0.25)),
    dict(seed=3, a=7.3, natoms=5, ecut_ry=12.0, lmax=2, k=(0.1, 0.2, -0.3)),
    dict(seed=4, a=np.array([[7.0, 0.0, 0.0], [1.1, 7.5, 0.0], [0.4, -0.6, 8.2]]), natoms=3,
         ecut_ry=12.0, lmax=1),
]


def system(cell, v):
    import paper_1709_10010_gb300 as pwh
    s = pwh.System.from_cell(cell)
    s.set_potential(v)
    return s


@pytest.mark.parametrize("kw", CASES)
def test_density_vs_oracle(torch, kw):
    cell, b, v, beta, D = case(**kw)
    s = system(cell, v)
    nb = 11
    psi = syn.initial_bands(5, b.npw, nb)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    occ = np.linspace(2.0, 0.0, nb)
    rho = s.density(torch.from_numpy(psi).cuda(), occ).cpu().numpy()
    ref = oscf.density(b.miller, b.fft, psi, occ, cell.volume)
    assert rel_err(rho, ref) <= 1e-12
    assert abs(rho.sum() * cell.volume / rho.size - occ.sum()) <= 1e-11


@pytest.mark.parametrize("kw", CASES)
def test_hartree_xc_vs_oracle(torch, kw):
    cell, b, v, beta, D = case(**kw)
    s = system(cell, v)
    psi = syn.initial_bands(6, b.npw, 8)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    rho = oscf.density(b.miller, b.fft, psi, np.full(8, 2.0), cell.volume)
    vt, en = s.hartree_xc(torch.from_numpy(rho).cuda(), torch.from_numpy(v).cuda())
    ref, en_ref = oscf.new_potential(cell.lattice, rho, v)
    assert rel_err(vt.cpu().numpy(), ref) <= 1e-12
    for k in en_ref:
        assert abs(en[k] - en_ref[k]) <= 1e-12 * max(1.0, abs(en_ref[k])), k
    # without the ionic part: V_H + v_xc alone
    vt0, _ = s.hartree_xc(torch.from_numpy(rho).cuda())
    ref0, _ = oscf.new_potential(cell.lattice, rho)
    assert rel_err(vt0.cpu().numpy(), ref0) <= 1e-12


def test_scf_steps_medium_cell(torch):
    """The 34,265-plane-wave cell (90^3 box, a compiled size): 64 bands."""
    cell = syn.config_cell("medium", 0)
    from oracle import basis as ob
    b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
    v = syn.potential_grid(cell, b.fft)
    s = system(cell, v)
    psi = syn.initial_bands(7, b.npw, 64)
    psi /= np.linalg.norm(psi, axis=1, keepdims=True)
    occ = np.full(64, 2.0)
    rho = s.density(torch.from_numpy(psi).cuda(), occ)
    ref = oscf.density(b.miller, b.fft, psi, occ, cell.volume)
    assert rel_err(rho.cpu().numpy(), ref) <= 1e-12
    vt, en = s.hartree_xc(rho, torch.from_numpy(v).cuda())
    vref, en_ref = oscf.new_potential(cell.lattice, ref, v)
    assert rel_err(vt.cpu().numpy(), vref) <= 1e-12
    assert abs(en["e_hartree"] - en_ref["e_hartree"]) <= 1e-11 * en_ref["e_hartree"]


def test_density_edge_cases(torch):
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(seed=1)
    s = system(cell, v)
    empty = torch.zeros((0, b.npw), dtype=torch.complex128, device="cuda")
    rho = s.density(empty, np.zeros(0))
    assert float(rho.abs().max()) == 0.0
    # null band block or output: an argument error, nothing launched
    assert pwh.lib().pwh_density(s._h, 2, None, b.npw, None, None) == 1
