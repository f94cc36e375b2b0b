"""Pins of the oracle's learned-preconditioner network (CPU only): central
finite differences, closed forms of degenerate networks, the Adam update rule,
and the feature/target definitions on constructed data."""
import math

import numpy as np

from oracle import mlp as om


def data(seed, rows=50):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((rows, 4))
    y = rng.standard_normal(rows)
    w = rng.uniform(0.1, 1.0, rows)
    return F, y, w


def test_gradient_matches_central_differences():
    p = om.init_params(1)
    p[-1] = 0.3
    p += 0.05 * np.random.default_rng(2).standard_normal(p.size)
    F, y, w = data(3)
    g = om.grad(p, F, y, w)
    h = 1e-6
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(p.size, 60, replace=False), [p.size - 1, 0, 300]])
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (om.loss(p + e, F, y, w) - om.loss(p - e, F, y, w)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 33)
    assert abs(om.silu(0.0)) == 0.0
    assert abs(om.silu(30.0) - 30.0) < 1e-10
    fd = (om.silu(z + 1e-6) - om.silu(z - 1e-6)) / 2e-6
    assert np.abs(fd - om.silu_grad(z)).max() < 1e-8


def test_constant_network_closed_form():
    """With zero output weights s = b3 for every row; dL/db3 = 2 sum w (b3 - y) / sum w
    and the other gradients of the output layer follow."""
    W1, b1, W2, b2, W3, b3 = om.unpack(om.init_params(5))
    p = om.pack(W1, b1, W2, b2, np.zeros_like(W3), np.array([0.7]))
    F, y, w = data(6)
    s, _ = om.forward(p, F)
    assert np.allclose(s, 0.7)
    g = om.grad(p, F, y, w)
    gb3 = g[-1]
    assert abs(gb3 - 2 * np.sum(w * (0.7 - y)) / np.sum(w)) < 1e-14
    gW1, gb1, gW2, gb2, gW3, _ = om.unpack(g)
    assert np.abs(gW1).max() == 0 and np.abs(gW2).max() == 0   # no path through W3 = 0


def test_adam_first_step_is_signed_learning_rate():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = om.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), rtol=0, atol=1e-15)


def test_training_reduces_loss():
    rng = np.random.default_rng(8)
    F = rng.standard_normal((400, 4))
    y = 0.5 * F[:, 0] - 0.3 * np.tanh(F[:, 2]) + 0.1
    w = np.ones(400)
    p = om.init_params(9)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = om.loss(p, F, y, w)
    for t in range(1, 301):
        p, m, v = om.adam_step(p, om.grad(p, F, y, w), m, v, t, lr=3e-3)
    assert om.loss(p, F, y, w) < 0.05 * l0


def test_features_closed_form():
    T = np.array([0.0, 2.0])
    f = om.features(T, theta=np.array([-0.5]), rnorm=np.array([1e-3]), eref=np.array([1.0]), vbar=-1.0)
    assert f.shape == (2, 4)
    np.testing.assert_allclose(f[0], [math.log(0.05), 0.5, -3.0, (0.0 - 1.0 + 0.5) / 1.0])
    np.testing.assert_allclose(f[1], [math.log(2.05), 0.5, -3.0, (2.0 - 1.0 + 0.5) / 3.0])


def test_targets_recover_a_planted_diagonal():
    """If the exact correction is e = -d_g r on every shell, the target is
    log d_g - log K_TPA minus the band's weighted mean."""
    rng = np.random.default_rng(10)
    nshell, npw, nb = 5, 60, 2
    shell = rng.integers(0, nshell, npw)
    T = np.linspace(0.0, 3.0, nshell)
    d = np.array([[0.5, 1.0, 2.0, 0.25, 3.0], [1.5, 0.2, 0.7, 1.1, 0.9]])
    R = rng.standard_normal((npw, nb)) + 1j * rng.standard_normal((npw, nb))
    E = -d.T[shell] * R
    eref = np.array([1.3, 0.8])
    y, w = om.targets_from_corrections(shell, nshell, T, R, E, eref)
    y, w = y.reshape(nb, nshell), w.reshape(nb, nshell)
    x = T[None, :] / eref[:, None]
    raw = np.log(d) - np.log(om.tpa(x))
    for n in range(nb):
        present = np.isin(np.arange(nshell), shell)
        ww = w[n][present]
        assert abs(ww.sum() - 1.0) < 1e-12
        expect = raw[n][present] - np.sum(ww * raw[n][present])
        np.testing.assert_allclose(y[n][present], expect, atol=1e-12)
    # a shell where the correction points the wrong way gets weight 0
    E2 = E.copy()
    E2[shell == 2, 0] *= -1
    y2, w2 = om.targets_from_corrections(shell, nshell, T, R, E2, eref)
    assert w2.reshape(nb, nshell)[0, 2] == 0.0


def test_targets_closed_form_exact_correction():
    """Pin of the exact correction inside ``targets``: take orthonormal converged
    bands X* and Ritz vectors X = X* U + eps Z with Z orthogonal to span(X*).
    The projector on span(X*) maps X to X* U, so the exact correction is
    e = P* x - x = -eps Z, known in closed form.  With residuals built as
    R = eps Z / d_g per shell, the best per-shell factor is d_g (> 0), so the
    targets must equal log d_g - log K_TPA minus the band's weighted mean, with
    every present shell weighted.  A sign slip (x - P* x), a transposed
    projector or the projector's complement breaks one of these."""
    rng = np.random.default_rng(11)
    nshell, npw, nb, eps = 6, 80, 3, 1e-2
    shell = np.concatenate([np.arange(nshell), rng.integers(0, nshell, npw - nshell)])
    T = np.linspace(0.1, 4.0, nshell)
    M = rng.standard_normal((npw, npw)) + 1j * rng.standard_normal((npw, npw))
    Qf, _ = np.linalg.qr(M)
    Xstar = Qf[:, :nb]
    Z = Qf[:, nb:nb + nb] @ (rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb)))
    U, _ = np.linalg.qr(rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb)))
    X = Xstar @ U + eps * Z
    d = rng.uniform(0.2, 3.0, (nb, nshell))
    R = eps * Z / d.T[shell]
    eref = np.array([0.9, 1.4, 2.2])
    y, w = om.targets(shell, nshell, T, X, R, Xstar, eref)
    y, w = y.reshape(nb, nshell), w.reshape(nb, nshell)
    x = T[None, :] / eref[:, None]
    raw = np.log(d) - np.log(om.tpa(x))
    for n in range(nb):
        assert np.all(w[n] > 0)
        assert abs(w[n].sum() - 1.0) < 1e-12
        np.testing.assert_allclose(y[n], raw[n] - np.sum(w[n] * raw[n]), atol=1e-10)
    # the weights are the residual's share per shell
    den = np.array([[np.sum(np.abs(R[shell == g, n]) ** 2) for g in range(nshell)] for n in range(nb)])
    np.testing.assert_allclose(w, den / den.sum(axis=1, keepdims=True), rtol=1e-12)
