"""Pins of the FP64 network oracle: encoding closed forms, a hand-computable network,
torch float64 autograd (a library restatement of the same network), FP64 central
finite differences (parameters and inputs), the loss against torch's library losses
and the Adam update against torch.optim.Adam."""

import math

import numpy as np
import pytest
import torch

from ddf_synth import init_weights
from oracle import mlp


def test_encoding_closed_form():
    o = np.array([[0.0, 0.5, 1.0]])
    w = np.array([[-0.5, -1.0, 0.25]])
    X, dX = mlp.encode(o, w, 4)
    assert X.shape == (1, 30)
    v = [0.0, 0.5, 1.0, -0.5, -1.0, 0.25]
    assert np.allclose(X[0, :6], v)
    s0 = np.array([0, 1, 0, -1, 0, math.sqrt(0.5)])        # sin(pi v)
    c0 = np.array([1, 0, -1, 0, -1, math.sqrt(0.5)])       # cos(pi v)
    s1 = np.array([0, 0, 0, 0, 0, 1])                      # sin(2 pi v)
    c1 = np.array([1, -1, 1, -1, 1, 0])                    # cos(2 pi v)
    assert np.allclose(X[0, 6:12], s0, atol=1e-15)
    assert np.allclose(X[0, 12:18], c0, atol=1e-15)
    assert np.allclose(X[0, 18:24], s1, atol=1e-15)
    assert np.allclose(X[0, 24:30], c1, atol=1e-15)
    # derivative columns: d sin(f v)/dv = f cos(f v)
    assert np.allclose(dX[0, 6:12], math.pi * c0, atol=1e-14)
    assert np.allclose(dX[0, 24:30], -2 * math.pi * s1, atol=1e-14)


def test_hand_network():
    # 6 -> 1 hidden unit -> 2, z = o_x + 0.5, y = (2 a + 0.1, -3 a + 0.2)
    blob = np.array([1, 0, 0, 0, 0, 0, 0.5, 2, -3, 0.1, 0.2], np.float64)
    P = mlp.unpack(blob, 0, 1, 1)
    o = np.array([[0.3, 0.1, 0.2], [-0.7, 0.0, 0.0]])
    w = np.array([[0.0, 0.0, -1.0], [1.0, 0.0, 0.0]])
    q = mlp.query(P, o, w, 0)
    assert np.allclose(q["dist"], [1.7, 0.1]) and np.allclose(q["logit"], [-2.2, 0.2])
    assert np.allclose(q["grad"][0], [2, 0, 0, 0, 0, 0]) and np.allclose(q["grad"][1], 0)
    assert np.allclose(q["normal"][0], [1, 0, 0])     # g . w = 0 -> kappa = +1
    assert np.allclose(q["normal"][1], [-1, 0, 0])    # zero gradient -> -w
    assert q["hit"].tolist() == [False, True]


def test_normal_orientation_rule():
    g = np.array([[0.0, 0.0, 2.0], [0.0, 0.0, -2.0], [3.0, 4.0, 0.0]])
    w = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    n = mlp.normal_from_gradient(g, w)
    assert np.allclose(n, [[0, 0, -1], [0, 0, -1], [0.6, 0.8, 0]])


def _torch_net(P, X):
    a = X
    for W, b in P[:-1]:
        a = torch.relu(a @ W.T + b)
    W, b = P[-1]
    return a @ W.T + b


def _torch_encode(o, w, F):
    v = torch.cat([o, w], 1)
    feats = [v]
    for k in range(F // 2):
        f = (2.0 ** k) * math.pi
        feats += [torch.sin(f * v), torch.cos(f * v)]
    return torch.cat(feats, 1)


@pytest.mark.parametrize("F,W,L", [(0, 64, 4), (12, 32, 3), (4, 16, 1)])
def test_against_torch_autograd(F, W, L):
    blob = init_weights(F, W, L, seed=7)
    P = mlp.unpack(blob, F, W, L)
    rng = np.random.default_rng(2)
    n = 257
    o = rng.uniform(-1, 1, (n, 3))
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    dist_gt = rng.uniform(0, 2, n)
    hit_gt = (rng.random(n) < 0.4).astype(np.uint8)
    # oracle
    L_o, grads, y = mlp.param_gradient(P, o, w, F, dist_gt, hit_gt)
    _, gin = mlp.input_gradient(P, o, w, F)
    # torch float64
    TP = [(torch.tensor(Wm, requires_grad=True), torch.tensor(b, requires_grad=True)) for Wm, b in P]
    to = torch.tensor(o, requires_grad=True)
    tw = torch.tensor(w, requires_grad=True)
    yt = _torch_net(TP, _torch_encode(to, tw, F))
    assert np.allclose(yt.detach().numpy(), y, rtol=1e-12, atol=1e-12)
    gx = torch.autograd.grad(yt[:, 0].sum(), [to, tw], retain_graph=True)
    assert np.allclose(torch.cat(gx, 1).numpy(), gin, rtol=1e-10, atol=1e-12)
    h = torch.tensor(hit_gt, dtype=torch.float64)
    m = h > 0
    l1 = torch.nn.functional.l1_loss(yt[m, 0], torch.tensor(dist_gt)[m], reduction="mean")
    bce = torch.nn.functional.binary_cross_entropy_with_logits(yt[:, 1], h, reduction="mean")
    loss = l1 + bce
    assert abs(loss.item() - L_o) < 1e-12
    tg = torch.autograd.grad(loss, [t for pair in TP for t in pair])
    for (dW, db), a, b in zip(grads, tg[0::2], tg[1::2]):
        assert np.allclose(dW, a.numpy(), rtol=1e-10, atol=1e-13)
        assert np.allclose(db, b.numpy(), rtol=1e-10, atol=1e-13)


def _mask_sig(P, X):
    _, pres, _ = mlp.forward(P, X)
    return np.concatenate([(z > 0) for z in pres], axis=1)


def test_param_gradient_finite_differences():
    """Central FP64 differences of the loss along random parameter directions and single
    coordinates, on a 1,024-ray subset of a 12-frequency 8 x 256 network (the training shape);
    rays whose ReLU pattern changes between the +h and -h passes are excluded."""
    F, W, L = 12, 256, 8
    blob = init_weights(F, W, L, seed=2).astype(np.float64)
    P = mlp.unpack(blob, F, W, L)
    rng = np.random.default_rng(11)
    n = 1024
    o = rng.normal(size=(n, 3))
    o /= np.linalg.norm(o, axis=1, keepdims=True)
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    dist_gt = rng.uniform(0, 2, n)
    hit_gt = (rng.random(n) < 0.5).astype(np.uint8)
    L0, grads, _ = mlp.param_gradient(P, o, w, F, dist_gt, hit_gt)
    g = mlp.pack(grads)
    X, _ = mlp.encode(o, w, F)
    h = 1e-6
    checked = 0
    for k in range(16 + 24):
        if k < 16:
            v = rng.normal(size=blob.size)
            v /= np.linalg.norm(v)
        else:
            v = np.zeros(blob.size)
            v[rng.integers(blob.size)] = 1.0
        Pp, Pm = mlp.unpack(blob + h * v, F, W, L), mlp.unpack(blob - h * v, F, W, L)
        keep = np.all(_mask_sig(Pp, X) == _mask_sig(Pm, X), axis=1)
        # rays whose L1 sign flips between the passes are also kinks
        yp, _, _ = mlp.forward(Pp, X)
        ym, _, _ = mlp.forward(Pm, X)
        keep &= (np.sign(yp[:, 0] - dist_gt) == np.sign(ym[:, 0] - dist_gt)) | (hit_gt == 0)
        if keep.sum() < n:
            continue
        lp, _ = mlp.loss_and_output_grad(yp, dist_gt, hit_gt)
        lm, _ = mlp.loss_and_output_grad(ym, dist_gt, hit_gt)
        fd = (lp - lm) / (2 * h)
        an = float(g @ v)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-8, (k, fd, an)
        checked += 1
    assert checked >= 30


def test_input_gradient_finite_differences():
    F, W, L = 12, 64, 4
    P = mlp.unpack(init_weights(F, W, L, seed=4), F, W, L)
    rng = np.random.default_rng(3)
    n = 256
    o = rng.uniform(-0.8, 0.8, (n, 3))
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    _, g = mlp.input_gradient(P, o, w, F)
    h = 1e-6
    X, _ = mlp.encode(o, w, F)
    sig0 = _mask_sig(P, X)
    v = np.concatenate([o, w], 1)
    ok_total = 0
    for j in range(6):
        vp, vm = v.copy(), v.copy()
        vp[:, j] += h
        vm[:, j] -= h
        Xp, _ = mlp.encode(vp[:, :3], vp[:, 3:], F)
        Xm, _ = mlp.encode(vm[:, :3], vm[:, 3:], F)
        keep = np.all(_mask_sig(P, Xp) == _mask_sig(P, Xm), axis=1) & np.all(_mask_sig(P, Xp) == sig0, axis=1)
        yp, _, _ = mlp.forward(P, Xp)
        ym, _, _ = mlp.forward(P, Xm)
        fd = (yp[:, 0] - ym[:, 0]) / (2 * h)
        assert np.allclose(fd[keep], g[keep, j], rtol=1e-5, atol=1e-7)
        ok_total += keep.sum()
    assert ok_total > 0.95 * 6 * n


def test_adam_against_torch():
    rng = np.random.default_rng(0)
    w0 = rng.normal(size=100)
    tw = torch.tensor(w0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tw], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    w, m, v = w0.copy(), np.zeros(100), np.zeros(100)
    for step in range(1, 6):
        g = rng.normal(size=100)
        tw.grad = torch.tensor(g)
        opt.step()
        w, m, v = mlp.adam_update(w, g, m, v, step, 1e-3, 0.9, 0.999, 1e-8)
        assert np.allclose(w, tw.detach().numpy(), rtol=0, atol=1e-15)
