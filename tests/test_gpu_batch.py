"""Batched eigensolves (pwh_batch_davidson_solve): many independent systems
(cells x k-points) solved concurrently give the same eigenvalues as one at a
time and as brute-force diagonalisation."""
import numpy as np
import pytest

from oracle import basis as ob
from oracle import hamiltonian as oh
from paper_1709_10010_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    from paper_1709_10010_gb300 import build
    build.build()
    return torch


def load(torch, cell):
    import paper_1709_10010_gb300 as pwh
    stream = torch.cuda.Stream()
    s = pwh.System.from_cell(cell, precision="mixed", stream=stream.cuda_stream)
    s._stream_keepalive = stream
    s.set_potential(syn.potential_grid(cell, s.fft))
    s.set_projectors(syn.projectors(cell, s.miller()), syn.d_diagonal(cell))
    return s


def test_batched_cells_and_kpoints_match_dense(torch):
    import paper_1709_10010_gb300 as pwh
    work = syn.batched_workload(ncells=2, seed=1, ecut_ry=12.0)     # 16 systems, small cutoff
    systems, psis, refs = [], [], []
    for cell, nb in work:
        s = load(torch, cell)
        nb = min(nb, 20)
        systems.append(s)
        psis.append(torch.from_numpy(syn.initial_bands(3, s.npw, nb)).cuda())
        b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
        H = oh.dense_h(b, syn.potential_grid(cell, b.fft), syn.projectors(cell, b.miller),
                       syn.d_diagonal(cell))
        refs.append(np.linalg.eigvalsh(H)[:nb])
    torch.cuda.synchronize()
    eigs, stats, status, st = pwh.batch_davidson(systems, psis, tol=1e-9, nthreads=8)
    assert st == 0 and all(x == 0 for x in status)
    for e, r in zip(eigs, refs):
        assert np.abs(e - r).max() <= 1e-8
    # the k-point pairs k, -k of one cell have the same spectrum (time reversal)
    assert np.abs(eigs[0] - eigs[7]).max() <= 1e-8


def test_batched_equals_sequential(torch):
    import paper_1709_10010_gb300 as pwh
    work = syn.batched_workload(ncells=1, seed=2, ecut_ry=16.0)
    systems = [load(torch, c) for c, _ in work]
    nb = 24
    starts = [syn.initial_bands(5, s.npw, nb) for s in systems]
    seq = []
    for s, p0 in zip(systems, starts):
        e, _, status = s.davidson(torch.from_numpy(p0).cuda(), tol=1e-9, mixed=True,
                                  switch_tol=1e-3, jd_inner=20)
        seq.append(e)
    psis = [torch.from_numpy(p0).cuda() for p0 in starts]
    torch.cuda.synchronize()
    eigs, stats, status, st = pwh.batch_davidson(systems, psis, tol=1e-9, nthreads=8)
    assert st == 0
    for a, b in zip(eigs, seq):
        assert np.abs(a - b).max() <= 1e-9


def test_batched_workload_30ry_subset_vs_dense(torch):
    """The batched workload's own shape (cells a ~ U(8,14) bohr, 4-16 atoms,
    s,p,d projectors, 30 Ry, the eight k-points of the 2x2x2 Monkhorst-Pack
    grid, the workload's band counts): its two smallest cells, 16 systems,
    solved together to 1e-8 in mixed precision + Jacobi-Davidson; every
    eigenvalue against brute-force diagonalisation of the oracle's H."""
    import paper_1709_10010_gb300 as pwh
    work = syn.batched_workload(ncells=32, seed=0)
    cells = {}
    for i, (cell, nb) in enumerate(work):
        cells.setdefault(i // 8, []).append((cell, nb))
    sizes = {c: ob.sphere(v[0][0].lattice, v[0][0].kpoint, v[0][0].ecut_ha).npw for c, v in cells.items()}
    pick = sorted(sizes, key=sizes.get)[:2]
    systems, psis, refs = [], [], []
    for c in pick:
        for j, (cell, nb) in enumerate(cells[c]):
            s = load(torch, cell)
            systems.append(s)
            psis.append(torch.from_numpy(syn.initial_bands(100 + 8 * c + j, s.npw, nb)).cuda())
            b = ob.sphere(cell.lattice, cell.kpoint, cell.ecut_ha)
            H = oh.dense_h(b, syn.potential_grid(cell, b.fft), syn.projectors(cell, b.miller),
                           syn.d_diagonal(cell))
            refs.append(np.linalg.eigvalsh(H)[:nb])
    torch.cuda.synchronize()
    eigs, stats, status, st = pwh.batch_davidson(systems, psis, tol=1e-8, switch_tol=1e-3,
                                                  jd_inner=20, nthreads=16)
    assert st == 0 and all(x == 0 for x in status)
    for e, r in zip(eigs, refs):
        assert np.abs(e - r).max() <= 1e-8
