"""Learned preconditioner of the oracle (TEST INFRASTRUCTURE; see
``oracle/__init__``).

Not in the paper: the learned part of the build.  A small network corrects
the Teter-Payne-Allan diagonal per (shell of equal |k+G|, band):

    K_MLP(G, n) = K_TPA(x) * exp(clip(s, -3, 3)),   s = MLP(f(shell(G), n))

MLP: 4 -> 64 -> 64 -> 1, SiLU(z) = z / (1 + exp(-z)) after both hidden
layers, linear output.  Parameters in one flat vector, in this order:
W1 (64x4, row-major), b1 (64), W2 (64x64), b2 (64), W3 (1x64), b3 (1).

Features of a (shell g, band n) pair, from the band's Ritz value theta_n,
residual norm ||r_n||, reference kinetic energy E_n = <x_n|T|x_n>, the shell's
kinetic energy T_g and the mean local potential vbar:

    x  = T_g / E_n
    f1 = log(x + 0.05)
    f2 = (theta_n - vbar) / E_n
    f3 = clip(log10 ||r_n||, -12, 2)
    f4 = (T_g + vbar - theta_n) / (T_g + E_n)

Target (from a Davidson trajectory and the converged bands X*): the exact
correction of band n is e_n = P* x_n - x_n with P* the projector on span(X*)
(well defined inside degenerate clusters).  Per shell, d_g = -<r,e>_g/<r,r>_g
is the best diagonal factor mapping the residual onto the correction (its
sign convention makes d_g ~ 1/(T_g - theta) > 0 where the kinetic term
dominates).  Rows with d_g > 0 get y = log d_g - log K_TPA(x) minus the
band's weighted mean (a per-band factor does not change the Davidson search
space), weight w = <r,r>_g / <r,r>; rows with d_g <= 0 get weight 0.

Loss: L = sum w (s - y)^2 / sum w.  Optimiser: Adam (Kingma & Ba, 2015) with
bias correction.
"""
from __future__ import annotations

import numpy as np

H1 = H2 = 64
NIN = 4
NPARAM = H1 * NIN + H1 + H2 * H1 + H2 + H2 + 1


def init_params(seed: int) -> np.ndarray:
    """Seeded initial parameters: weights ~ N(0, 1/fan_in), biases 0, output 0."""
    rng = np.random.default_rng([int(seed), 7])
    W1 = rng.standard_normal((H1, NIN)) / np.sqrt(NIN)
    W2 = rng.standard_normal((H2, H1)) / np.sqrt(H1)
    W3 = rng.standard_normal((1, H2)) / np.sqrt(H2) * 0.1
    return pack(W1, np.zeros(H1), W2, np.zeros(H2), W3, np.zeros(1))


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H1 * NIN].reshape(H1, NIN); o += H1 * NIN
    b1 = p[o:o + H1]; o += H1
    W2 = p[o:o + H2 * H1].reshape(H2, H1); o += H2 * H1
    b2 = p[o:o + H2]; o += H2
    W3 = p[o:o + H2].reshape(1, H2); o += H2
    b3 = p[o:o + 1]
    return W1, b1, W2, b2, W3, b3


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


def forward(p, F):
    """s for every row of F (rows, 4), plus the cache for backward."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    z1 = F @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    s = (h2 @ W3.T + b3)[:, 0]
    return s, (F, z1, h1, z2, h2)


def loss(p, F, y, w):
    s, _ = forward(p, F)
    return float(np.sum(w * (s - y) ** 2) / np.sum(w))


def grad(p, F, y, w):
    """dL/dp by reverse-mode differentiation of the layers above."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    s, (F, z1, h1, z2, h2) = forward(p, F)
    ds = 2.0 * w * (s - y) / np.sum(w)            # (rows,)
    gW3 = ds[None, :] @ h2                          # (1, 64)
    gb3 = np.array([ds.sum()])
    dh2 = ds[:, None] * W3                          # (rows, 64)
    dz2 = dh2 * silu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * silu_grad(z1)
    gW1 = dz1.T @ F
    gb1 = dz1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def tpa(x):
    q = 27.0 + 18.0 * x + 12.0 * x ** 2 + 8.0 * x ** 3
    return q / (q + 16.0 * x ** 4)


def features(T_shell, theta, rnorm, eref, vbar):
    """Rows (nshell * nb, 4), shell-major within each band: row = n * nshell + g."""
    Tg = np.asarray(T_shell)[None, :]
    th = np.asarray(theta)[:, None]
    E = np.asarray(eref)[:, None]
    x = Tg / E
    f1 = np.log(x + 0.05)
    f2 = np.broadcast_to((th - vbar) / E, x.shape)
    f3 = np.broadcast_to(np.clip(np.log10(np.asarray(rnorm))[:, None], -12, 2), x.shape)
    f4 = (Tg + vbar - th) / (Tg + E)
    return np.stack([f1, f2, f3, f4], axis=-1).reshape(-1, 4)


def targets(shell, nshell, T_shell, X, R, Xstar, eref):
    """(y, w) per row (n * nshell + g) from Ritz vectors X, residuals R and the
    converged bands Xstar (all (npw, nb) columns)."""
    E = Xstar @ (Xstar.conj().T @ X) - X            # exact corrections
    return targets_from_corrections(shell, nshell, T_shell, R, E, eref)


def targets_from_corrections(shell, nshell, T_shell, R, E, eref):
    nb = R.shape[1]
    num = np.zeros((nb, nshell))
    den = np.zeros((nb, nshell))
    for n in range(nb):
        np.add.at(num[n], shell, np.real(np.conj(R[:, n]) * E[:, n]))
        np.add.at(den[n], shell, np.abs(R[:, n]) ** 2)
    d = np.where(den > 0, -num / np.where(den > 0, den, 1.0), 0.0)
    x = np.asarray(T_shell)[None, :] / np.asarray(eref)[:, None]
    ok = (d > 0) & (den > 0)
    y = np.where(ok, np.log(np.where(ok, d, 1.0)) - np.log(tpa(x)), 0.0)
    w = np.where(ok, den / den.sum(axis=1, keepdims=True), 0.0)
    mean = (w * y).sum(axis=1, keepdims=True) / np.maximum(w.sum(axis=1, keepdims=True), 1e-300)
    y = np.where(ok, y - mean, 0.0)
    return y.reshape(-1), w.reshape(-1)
