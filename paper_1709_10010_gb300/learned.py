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
    bands.  Returns (F, y, w) CUDA tensors."""
    import torch
    nb = int(psi0.shape[0])
    if xstar is None:
        xstar = psi0.clone()
        _, _, st = system.davidson(xstar, tol=tol, mixed=True, switch_tol=1e-3, jd_inner=20,
                                   check=False)
    prec_saved = None
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
    del prec_saved
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
