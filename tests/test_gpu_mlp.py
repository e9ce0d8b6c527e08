"""Planner MLP kernels vs the fp64 oracle: forward, gradients (normwise per
tensor within 1e-4), one Adam step (1e-6), and training lowers the loss."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def setup(ctx, lh, n=300, n_in=60, hidden=64, seed=3):
    import torch
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n_in)).astype(np.float32)
    y = rng.normal(size=n).astype(np.float32)
    m = lh.Model(ctx, n_in, hidden, seed=seed)
    return m, X, y, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()


def test_forward_and_gradients_match_oracle(ctx, orc, lhlib):
    lh = lhlib
    m, X, y, dX, dy = setup(ctx, lh)
    P = {k: v.astype(np.float64) for k, v in lh.unpack_params(m.params(), 60, 64).items()}
    out = m.forward(dX).cpu().numpy()
    want, _ = orc.mlp_forward(P, X)
    assert np.allclose(out, want, rtol=1e-5, atol=1e-5)
    loss = m.loss_grad(dX, dy)
    wl, wg = orc.mlp_loss_grad(P, X, y)
    assert abs(loss - wl) <= 1e-5 * max(1.0, abs(wl))
    G = lh.unpack_params(m.grads(), 60, 64)
    for k in wg:
        g = G[k].astype(np.float64).reshape(wg[k].shape)
        assert np.linalg.norm(g - wg[k]) <= 1e-4 * max(np.linalg.norm(wg[k]), 1e-12), k
    m.free()


def test_adam_step_matches_oracle(ctx, orc, lhlib):
    lh = lhlib
    m, X, y, dX, dy = setup(ctx, lh, seed=5)
    p0 = m.params().astype(np.float64)
    m.loss_grad(dX, dy)
    g = m.grads().astype(np.float64)
    m.adam_step(lr=1e-3)
    P = {"w": p0.copy()}
    G = {"w": g}
    M = {"w": np.zeros_like(p0)}
    V = {"w": np.zeros_like(p0)}
    orc.adam_step(P, G, M, V, t=1, lr=1e-3)
    assert np.allclose(m.params(), P["w"], rtol=0, atol=1e-6)
    m.free()


def test_training_lowers_loss(ctx, lhlib):
    import torch
    lh = lhlib
    rng = np.random.default_rng(9)
    X = rng.normal(size=(2000, 60)).astype(np.float32)
    w = rng.normal(size=60)
    y = (np.tanh(X @ w / 8) + 0.1 * np.sin(X[:, 0])).astype(np.float32)
    dX, dy = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    m = lh.Model(ctx, 60, 64, seed=1)
    l0 = m.loss_grad(dX, dy)
    l1 = m.train(dX, dy, epochs=40, batch=128, lr=1e-3, seed=2)
    assert l1 < 0.2 * l0, (l0, l1)
    m.free()
