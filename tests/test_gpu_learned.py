"""The learned-preconditioner protocol on a reduced workload (the full one,
200 training cells of the 34k-plane-wave shape and 20 held-out seeds, runs
with ``python -m paper_1709_10010_gb300.learned``): training rows from FP64
Davidson trajectories of 6 small cells, full-batch Adam on the GPU, then TPA
against the trained network on 2 held-out cells, plain mixed-precision
Davidson (switch 1e-5, no Jacobi-Davidson: the outer preconditioner shapes
every search direction).  The test checks that training lowers the loss,
that every solve converges to the same eigenvalues (1e-9 Ha), and bounds the
network's iterations by 1.5x those of TPA; it prints the difference, which
the full protocol reports as the measured effect."""
import numpy as np
import pytest

from paper_1709_10010_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def small_cell(seed):
    rng = np.random.default_rng([seed, 13])
    return syn.make_cell(seed, float(rng.uniform(9.0, 11.0)), int(rng.integers(8, 13)), 16.0, 2)


def test_learned_preconditioner_reduced_protocol():
    import torch
    from paper_1709_10010_gb300 import build, learned
    build.build()
    nb = 24
    parts = []
    for seed in range(300, 306):
        s = learned.load_system(small_cell(seed))
        psi0 = torch.from_numpy(syn.initial_bands(seed, s.npw, nb)).cuda()
        F, y, w = learned.harvest(s, psi0, snapshots=(2, 5, 10))
        keep = torch.nonzero(w > 0).flatten()
        parts.append((F[keep], y[keep], w[keep]))
    rows = tuple(torch.cat([p[i] for p in parts]) for i in range(3))
    blob, hist = learned.train(s, rows, steps=800, lr=2e-3, log_every=200)
    assert hist[-1][1] < 0.5 * hist[0][1]
    it = {"tpa": 0, "mlp": 0}
    for seed in (400, 401):
        s = learned.load_system(small_cell(seed))
        s.set_mlp(blob)
        psi0 = torch.from_numpy(syn.initial_bands(seed, s.npw, nb)).cuda()
        eigs = {}
        for pc in ("tpa", "mlp"):
            eig, st, status = s.davidson(psi0.clone(), tol=1e-9, precond=pc, mixed=True,
                                         switch_tol=1e-5, jd_inner=0, max_iter=400)
            assert status == 0
            it[pc] += st["iters"]
            eigs[pc] = eig
        assert np.abs(eigs["tpa"] - eigs["mlp"]).max() <= 1e-9
    print(f"iterations on 2 held-out cells: TPA {it['tpa']}, learned {it['mlp']}")
    assert it["mlp"] <= 1.5 * it["tpa"]
