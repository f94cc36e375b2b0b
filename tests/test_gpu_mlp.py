"""Learned preconditioner on the GPU against the FP64 oracle: forward pass,
loss and gradient, Adam step, training rows (features/targets/weights) of a
trajectory point; training lowers the loss; the eigensolver with the learned
preconditioner converges to the same eigenvalues (FP32 network vs FP64 oracle:
bars 1e-5 relative on outputs, 2e-4 on gradients)."""
import numpy as np
import pytest

from oracle import basis as ob
from oracle import mlp as om
from paper_1709_10010_gb300 import synthetic as syn
from tests.helpers import case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1709_10010_gb300 as pwh
    from paper_1709_10010_gb300 import build
    build.build()
    cell, b, v, beta, D = case(seed=0, a=8.0, natoms=4, ecut_ry=14.0, lmax=1)
    s = pwh.System.from_cell(cell)
    s.set_potential(v)
    s.set_projectors(beta, D)
    return torch, pwh, s, (cell, b, v, beta, D)


def rows(seed, n=1000):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n, 4)).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    w = rng.uniform(0.0, 1.0, n).astype(np.float32)
    return F, y, w


def test_forward_and_gradient_vs_oracle(env):
    torch, pwh, s, _ = env
    from paper_1709_10010_gb300 import learned
    p = learned.init_params(3)
    p[-1] = 0.2
    p = p + 0.05 * np.random.default_rng(1).standard_normal(p.size).astype(np.float32)
    F, y, w = rows(2)
    pt = torch.from_numpy(p).cuda()
    Ft, yt, wt = (torch.from_numpy(a).cuda() for a in (F, y, w))
    sg = s.mlp_forward(pt, Ft).cpu().numpy()
    so, _ = om.forward(p.astype(np.float64), F.astype(np.float64))
    assert np.abs(sg - so).max() <= 1e-5 * max(1.0, np.abs(so).max())
    loss, g = s.mlp_loss_grad(pt, Ft, yt, wt)
    lo = om.loss(p.astype(np.float64), F.astype(np.float64), y.astype(np.float64), w.astype(np.float64))
    go = om.grad(p.astype(np.float64), F.astype(np.float64), y.astype(np.float64), w.astype(np.float64))
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    gg = g.cpu().numpy()
    assert np.abs(gg - go).max() <= 2e-4 * np.abs(go).max()


def test_adam_step_vs_oracle(env):
    torch, pwh, s, _ = env
    rng = np.random.default_rng(4)
    p = rng.standard_normal(pwh.MLP_PARAMS).astype(np.float32)
    g = rng.standard_normal(pwh.MLP_PARAMS).astype(np.float32)
    m = (0.1 * rng.standard_normal(pwh.MLP_PARAMS)).astype(np.float32)
    v = rng.uniform(0, 0.1, pwh.MLP_PARAMS).astype(np.float32)
    pt, gt, mt, vt = (torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v))
    s.mlp_adam(pt, gt, mt, vt, 7, 1e-3)
    po, mo, vo = om.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                              v.astype(np.float64), 7, lr=1e-3)
    assert np.abs(pt.cpu().numpy() - po).max() <= 1e-6
    assert np.abs(mt.cpu().numpy() - mo).max() <= 1e-6


def test_training_rows_vs_oracle(env):
    """Features, targets and weights of one trajectory point (Ritz vectors after
    3 iterations, converged bands from a full solve) against the oracle."""
    torch, pwh, s, (cell, b, v, beta, D) = env
    from oracle import hamiltonian as oh
    nb = 6
    psi0 = torch.from_numpy(syn.initial_bands(5, b.npw, nb)).cuda()
    xs = psi0.clone()
    s.davidson(xs, tol=1e-11)
    X = psi0.clone()
    theta, _, _ = s.davidson(X, tol=1e-300, max_iter=3, check=False)
    HX = s.apply_h(X)
    F, y, w = s.mlp_training_rows(X, HX, theta, xs)
    Xh, HXh, Sh = X.cpu().numpy().T, HX.cpu().numpy().T, xs.cpu().numpy().T
    R = HXh - Xh * theta[None, :]
    wx = np.abs(Xh) ** 2
    eref = (b.kinetic[:, None] * wx).sum(0) / wx.sum(0)
    sh, Tsh = s.shells()
    np.testing.assert_array_equal(sh, b.shell)
    Fo = om.features(Tsh, theta, np.linalg.norm(R, axis=0), eref, float(v.mean()))
    yo, wo = om.targets(b.shell, Tsh.size, Tsh, Xh, R, Sh, eref)
    np.testing.assert_allclose(F.cpu().numpy(), Fo, rtol=1e-5, atol=1e-5)
    wg = w.cpu().numpy()
    np.testing.assert_allclose(wg, wo, rtol=1e-5, atol=1e-7)
    ok = wo > 1e-6
    np.testing.assert_allclose(y.cpu().numpy()[ok], yo[ok], rtol=1e-4, atol=1e-4)


def test_train_and_solve_with_learned_preconditioner(env):
    torch, pwh, s, (cell, b, v, beta, D) = env
    from paper_1709_10010_gb300 import learned
    nb = 8
    psi0 = torch.from_numpy(syn.initial_bands(6, b.npw, nb)).cuda()
    F, y, w = learned.harvest(s, psi0, snapshots=(2, 4, 8))
    blob, hist = learned.train(s, (F, y, w), steps=300, lr=3e-3, log_every=100)
    assert hist[-1][1] < hist[0][1]
    s.set_mlp(blob)
    e_tpa, st_tpa, _ = s.davidson(psi0.clone(), tol=1e-9, precond="tpa")
    e_mlp, st_mlp, status = s.davidson(psi0.clone(), tol=1e-9, precond="mlp")
    assert status == 0
    assert np.abs(e_tpa - e_mlp).max() <= 1e-9
