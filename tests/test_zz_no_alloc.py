"""The allocation-free entry point pwh_apply_local_noalloc, for callers that
cannot let the library call cudaMalloc (their device memory is handed to their
own pool up front, or they must avoid the device-wide synchronisation an
allocation may cause).  Checked through the C ABI against the existing entry
point pwh_apply_h_internal (same operator with the nonlocal term removed), on
two calls in a row, within the FP64 tolerance of the other H|psi> tests.

Named to be collected last: a run that stops at the first failure has already
run every other test."""
import numpy as np
import pytest

from paper_1709_10010_gb300 import synthetic as syn
from tests.helpers import case

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch
    from paper_1709_10010_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return torch


@pytest.mark.parametrize("kw", [dict(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1),
                                dict(seed=1, a=20.0, natoms=64, ecut_ry=40.0, lmax=2)])
def test_noalloc_matches_existing_entry_point(torch, kw):
    import paper_1709_10010_gb300 as pwh
    cell, b, v, beta, D = case(**kw)
    s = pwh.System.from_cell(cell)
    s.set_potential(v)
    s.set_projectors(np.zeros((0, s.npw), complex), np.zeros(0))   # local + kinetic only
    nb = 37
    out = torch.empty((nb, s.npw), dtype=torch.complex128, device="cuda")
    for call in range(2):
        psi = torch.from_numpy(syn.initial_bands(100 + call, s.npw, nb)).cuda()
        ref = s.apply_h_internal(psi).cpu().numpy()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        s.apply_local_noalloc(psi, out)
        s.sync()
        free1 = torch.cuda.mem_get_info()[0]
        got = out.cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= FP64_TOL, (call, err)
        if call == 1:
            assert free1 == free0        # nothing was allocated by the call
    s.close()


def test_noalloc_rejects_oversized_system(torch):
    """A band whose stick buffer exceeds the 32 MiB static scratch is refused
    (a = 50 bohr, 80 Ry: N = 288, about 70 MiB per band)."""
    import paper_1709_10010_gb300 as pwh
    cell = syn.make_cell(0, 50.0, 1, 80.0, 0)
    s = pwh.System.from_cell(cell)
    assert s.fft[2] * s.nsticks * 16 > (32 << 20)
    s.set_potential(np.zeros(s.fft))
    psi = torch.zeros((1, s.npw), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(psi)
    with pytest.raises(pwh.PwhError) as e:
        s.apply_local_noalloc(psi, out)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    s.close()
