"""Training driver of the learned preconditioner (the network, its data and
its optimiser all run in libpwh's kernels; this module sequences the calls).

    rows = harvest(system, psi0, snapshots)      # (features, targets, weights) on the GPU
    blob = train(system, rows, steps=..., lr=...) # Adam on the GPU, full batch
    system.set_mlp(blob)                          # used by precond="mlp"

Training data come from the solver's own trajectories: the plain FP64 Davidson
is stopped after ``it`` iterations for each ``it`` in ``snapshots`` (the Ritz
vectors and values at that point), H X is applied in FP64, and the converged
bands X* of a full solve give the exact corrections.
"""
from __future__ import annotations

import numpy as np

from . import MLP_BLOB, MLP_PARAMS

HIDDEN = 64


def init_params(seed: int) -> np.ndarray:
    """Seeded start: weights ~ N(0, 1/fan_in) (output layer scaled by 0.1), biases 0."""
    rng = np.random.default_rng([int(seed), 11])
    W1 = rng.standard_normal((HIDDEN, 4)) / 2.0
    W2 = rng.standard_normal((HIDDEN, HIDDEN)) / 8.0
    W3 = rng.standard_normal(HIDDEN) / 8.0 * 0.1
    p = np.concatenate([W1.ravel(), np.zeros(HIDDEN), W2.ravel(), np.zeros(HIDDEN), W3, [0.0]])
    assert p.size == MLP_PARAMS
    return p.astype(np.float32)


def harvest(system, psi0, snapshots=(2, 5, 10, 20), xstar=None, tol=1e-8):
    """Training rows from one system.  psi0: (nb, npw) CUDA complex128 starting
    bands.  Returns (F, y, w) CUDA tensors.  Leaves the system's apply
    precision at FP64."""
    import torch
    nb = int(psi0.shape[0])
    if xstar is None:
        xstar = psi0.clone()
        _, _, st = system.davidson(xstar, tol=tol, mixed=True, switch_tol=1e-3, jd_inner=20,
                                   check=False)
    Fs, ys, ws = [], [], []
    for it in snapshots:
        X = psi0.clone()
        theta, _, _ = system.davidson(X, tol=1e-300, max_iter=int(it), mixed=False, check=False)
        system.set_precision("fp64")
        HX = system.apply_h(X)
        F, y, w = system.mlp_training_rows(X, HX, theta, xstar)
        Fs.append(F)
        ys.append(y)
        ws.append(w)
    return torch.cat(Fs), torch.cat(ys), torch.cat(ws)


def train(system, rows, steps=2000, lr=2e-3, seed=0, log_every=0):
    """Full-batch Adam on the GPU.  Returns (blob numpy float32 of MLP_BLOB
    entries, loss history)."""
    import torch
    F, y, w = rows
    wh = w.double().cpu().numpy()
    wsum = float(wh.sum())
    Fh = F.cpu().numpy()[wh > 0]
    lo, hi = Fh.min(axis=0), Fh.max(axis=0)
    p = torch.from_numpy(init_params(seed)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    hist = []
    for t in range(1, steps + 1):
        loss, g = system.mlp_loss_grad(p, F, y, w, wsum=wsum)
        system.mlp_adam(p, g, m, v, t, lr)
        if log_every and (t % log_every == 0 or t == 1):
            hist.append((t, float(loss.item())))
    loss, _ = system.mlp_loss_grad(p, F, y, w, wsum=wsum)
    hist.append((steps, float(loss.item())))
    blob = np.concatenate([p.cpu().numpy(), lo, hi]).astype(np.float32)
    assert blob.size == MLP_BLOB
    return blob, hist


def workload_cell(seed):
    """A cell of the learned-preconditioner workload: cubic a ~ U(16, 20) bohr,
    32-64 atoms, 40 Ry, s,p,d projectors (the shape of the 34k-plane-wave cell)."""
    from . import synthetic as syn
    rng = np.random.default_rng([int(seed), 3])
    a = float(rng.uniform(16.0, 20.0))
    natoms = int(rng.integers(32, 65))
    return syn.make_cell(seed, a, natoms, 40.0, 2)


def load_system(cell, precision="mixed"):
    import paper_1709_10010_gb300 as pwh
    from . import synthetic as syn
    s = pwh.System.from_cell(cell, precision=precision)
    s.set_potential(syn.potential_grid(cell, s.fft))
    s.set_projectors(syn.projectors(cell, s.miller()), syn.d_diagonal(cell))
    return s


def evaluate(blob, seeds, nb=128, modes=("mixed", "mixed_jd")):
    """Held-out comparison: for every seed, the same cell and start solved to
    1e-8 with the TPA and with the learned preconditioner, per solver mode.
    Returns one dict per seed (iterations, H applications, seconds, status,
    final residual, max |dlambda| between the two)."""
    import time

    import torch

    from . import synthetic as syn
    kws = {"mixed": dict(mixed=True, switch_tol=1e-5, jd_inner=0),
           "mixed_jd": dict(mixed=True, switch_tol=1e-3, jd_inner=20)}
    res = []
    for seed in seeds:
        s = load_system(workload_cell(seed))
        s.set_mlp(blob)
        psi0 = torch.from_numpy(syn.initial_bands(seed, s.npw, nb)).cuda()
        row = {"seed": int(seed), "npw": s.npw}
        eigs = {}
        for mode in modes:
            for pc in ("tpa", "mlp"):
                psi = psi0.clone()
                torch.cuda.synchronize()
                t = time.perf_counter()
                eig, st, status = s.davidson(psi, tol=1e-8, precond=pc, check=False, **kws[mode])
                torch.cuda.synchronize()
                row[f"{pc}_{mode}"] = {"iters": st["iters"], "n_apply": st["n_apply"],
                                       "time_s": time.perf_counter() - t, "status": status,
                                       "resid": st["max_resid"]}
                eigs[f"{pc}_{mode}"] = eig
            row[f"max_dlambda_{mode}"] = float(np.abs(eigs[f"tpa_{mode}"] - eigs[f"mlp_{mode}"]).max())
        res.append(row)
        s.close()
    return res


def summarize(res, modes=("mixed", "mixed_jd")):
    out = {}
    for mode in modes:
        it = {pc: sum(r[f"{pc}_{mode}"]["iters"] for r in res) for pc in ("tpa", "mlp")}
        tm = {pc: sum(r[f"{pc}_{mode}"]["time_s"] for r in res) for pc in ("tpa", "mlp")}
        out[mode] = {"iters_total": it, "time_total_s": tm,
                     "all_converged": all(r[f"{pc}_{mode}"]["status"] == 0
                                          for r in res for pc in ("tpa", "mlp")),
                     "max_dlambda_ha": max(r[f"max_dlambda_{mode}"] for r in res)}
    return out


def main():
    """The learned-preconditioner protocol: training rows from FP64 Davidson
    trajectories on --train cells (seeds 1000..), a random subset of about
    --rows rows, full-batch Adam on the GPU, then TPA vs MLP on --test
    held-out cells (seeds 2000..).  Prints one JSON record."""
    import argparse
    import json
    import time

    import torch

    from . import synthetic as syn
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--test", type=int, default=20)
    ap.add_argument("--nb", type=int, default=128)
    ap.add_argument("--rows", type=int, default=1_000_000)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--out", default=None, help="save the trained blob (.npy)")
    ap.add_argument("--eval-only", default=None, metavar="BLOB",
                    help="skip harvesting and training: evaluate this saved blob (.npy)")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    if a.eval_only:
        blob = np.load(a.eval_only).astype(np.float32)
        res = evaluate(blob, range(2000, 2000 + a.test), nb=a.nb)
        print(json.dumps({"test_cells": a.test, "nb": a.nb, "blob": a.eval_only,
                          "summary": summarize(res), "held_out": res}))
        return
    t0 = time.time()
    parts, nrows = [], 0
    s = None
    for seed in range(1000, 1000 + a.train):
        s = load_system(workload_cell(seed))
        psi0 = torch.from_numpy(syn.initial_bands(seed, s.npw, a.nb)).cuda()
        F, y, w = harvest(s, psi0, snapshots=(2, 5, 10))
        keep = torch.nonzero(w > 0).flatten()
        parts.append((F[keep], y[keep], w[keep]))
        nrows += int(keep.numel())
        s.close()
    F = torch.cat([p[0] for p in parts])
    y = torch.cat([p[1] for p in parts])
    w = torch.cat([p[2] for p in parts])
    if F.shape[0] > a.rows:
        g = torch.Generator(device="cuda").manual_seed(0)
        pick = torch.randperm(F.shape[0], device="cuda", generator=g)[:a.rows]
        F, y, w = F[pick], y[pick], w[pick]
    t_data = time.time() - t0
    s = load_system(workload_cell(1000))
    blob, hist = train(s, (F, y, w), steps=a.steps, lr=2e-3, log_every=500)
    s.close()
    t_train = time.time() - t0 - t_data
    if a.out:
        np.save(a.out, blob)
    res = evaluate(blob, range(2000, 2000 + a.test), nb=a.nb)
    print(json.dumps({"train_cells": a.train, "test_cells": a.test, "nb": a.nb,
                      "rows_harvested": nrows, "rows_trained": int(F.shape[0]),
                      "data_s": t_data, "train_s": t_train, "loss_history": hist,
                      "summary": summarize(res), "held_out": res}))


if __name__ == "__main__":
    main()
