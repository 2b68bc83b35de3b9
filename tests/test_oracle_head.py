"""Pins of the single-output head, the clamp and squish losses and weight normalisation
(oracle/head.py) against torch float64 autograd: torch.clamp / torch.tanh losses, torch's own
weight-norm parametrisation, and a whole single-output network written in torch, whose parameter
gradients the oracle's pieces (forward, loss, reverse pass, weight-norm chain rule) must
reproduce."""

import numpy as np
import pytest
import torch

from oracle import head as H
from oracle import mlp as omlp


def _outputs(n, delta, seed):
    rng = np.random.default_rng(seed)
    d = rng.uniform(-1.5 * delta, 2.0 * delta, n)
    hit = (rng.random(n) < 0.6).astype(np.uint8)
    dgt = rng.uniform(0.0, 2.0 * delta, n)
    # stay off the kinks (|x|'s at 0, the clamp's at +-delta)
    bad = (np.abs(np.abs(d) - delta) < 1e-3) | (np.abs(np.minimum(delta, np.maximum(-delta, d))
                                                       - np.where(hit > 0, np.minimum(dgt, delta), delta)) < 1e-3)
    d[bad] += 3e-3
    y = np.stack([d, rng.normal(size=n)], 1)
    return y, dgt, hit


def _torch_target(dgt, hit):
    return torch.where(torch.from_numpy(hit > 0), torch.from_numpy(dgt), torch.tensor(float("inf"), dtype=torch.float64))


@pytest.mark.parametrize("delta", [0.1, 0.5])
def test_clamp_loss_matches_torch(delta):
    y, dgt, hit = _outputs(4000, delta, 1)
    L, gy = H.clamp_loss_and_output_grad(y, dgt, hit, delta)
    d = torch.from_numpy(y[:, 0].copy()).requires_grad_(True)
    ref = torch.mean(torch.abs(torch.clamp(_torch_target(dgt, hit), -delta, delta) - torch.clamp(d, -delta, delta)))
    ref.backward()
    assert abs(L - ref.item()) < 1e-13
    assert np.allclose(gy[:, 0], d.grad.numpy(), rtol=0, atol=1e-15)
    assert (gy[:, 1] == 0).all()
    assert (gy[np.abs(y[:, 0]) > delta, 0] == 0).all() and (gy[np.abs(y[:, 0]) < delta, 0] != 0).mean() > 0.99


def test_squish_loss_matches_torch():
    y, dgt, hit = _outputs(4000, 0.8, 2)
    L, gy = H.squish_loss_and_output_grad(y, dgt, hit)
    d = torch.from_numpy(y[:, 0].copy()).requires_grad_(True)
    ref = torch.mean(torch.abs(torch.tanh(_torch_target(dgt, hit)) - torch.tanh(d)))
    ref.backward()
    assert abs(L - ref.item()) < 1e-13
    assert np.allclose(gy[:, 0], d.grad.numpy(), rtol=1e-12, atol=1e-16)


def test_weight_norm_matches_torch_parametrisation():
    rng = np.random.default_rng(3)
    W = rng.normal(size=(64, 40))
    R = rng.normal(size=(64, 40))                     # an upstream gradient of the folded weight
    v, g = H.wn_init(W)
    assert np.allclose(H.wn_fold(v, g), W, rtol=1e-14, atol=1e-15)
    lin = torch.nn.Linear(40, 64, bias=False).double()
    with torch.no_grad():
        lin.weight.copy_(torch.from_numpy(W))
    lin = torch.nn.utils.parametrizations.weight_norm(lin, dim=0)
    g_t = lin.parametrizations.weight.original0       # (64, 1)
    v_t = lin.parametrizations.weight.original1       # (64, 40)
    assert np.allclose(g_t.detach().numpy()[:, 0], g, rtol=1e-14)
    assert np.allclose(v_t.detach().numpy(), v)
    # move away from v = W so that |v| != g
    v2 = v * rng.uniform(0.5, 2.0, size=(64, 1)) + 0.1 * rng.normal(size=v.shape)
    g2 = g * rng.uniform(0.5, 1.5, size=64)
    with torch.no_grad():
        v_t.copy_(torch.from_numpy(v2))
        g_t.copy_(torch.from_numpy(g2)[:, None])
    assert np.allclose(lin.weight.detach().numpy(), H.wn_fold(v2, g2), rtol=1e-13, atol=1e-15)
    (lin.weight * torch.from_numpy(R)).sum().backward()
    dv, dg = H.wn_grad(v2, g2, R)
    assert np.allclose(dv, v_t.grad.numpy(), rtol=1e-11, atol=1e-13)
    assert np.allclose(dg, g_t.grad.numpy()[:, 0], rtol=1e-11, atol=1e-13)


def test_derived_head_gives_logit_delta_minus_y():
    rng = np.random.default_rng(4)
    params = [(rng.normal(size=(32, 18)) * 0.3, rng.normal(size=32) * 0.1),
              (rng.normal(size=(32, 32)) * 0.3, rng.normal(size=32) * 0.1),
              (rng.normal(size=(2, 32)) * 0.3, rng.normal(size=2))]
    p2 = H.derive_single_head(params, 0.25)
    X = rng.normal(size=(500, 18))
    y, _, _ = omlp.forward(p2, X)
    y0, _, _ = omlp.forward(params, X)
    assert np.array_equal(y[:, 0], y0[:, 0])                       # row 0 untouched
    assert np.allclose(y[:, 1], 0.25 - y[:, 0], rtol=0, atol=1e-14)
    assert np.array_equal(y[:, 1] > 0, y[:, 0] < 0.25)


@pytest.mark.parametrize("loss", ["clamp", "squish"])
def test_single_output_network_gradient_matches_torch(loss):
    """A whole single-output, weight-normalised network in torch (hidden Linear layers under
    torch's weight-norm parametrisation, a 1-output head): the oracle's forward on the derived
    head, its loss gradient, its reverse pass and the weight-norm chain rule give the same loss
    and the same gradients of every v, g, bias and the head's row."""
    rng = np.random.default_rng(5)
    F, Wd, L, delta = 2, 24, 3, 0.4
    E = 6 + 6 * F
    n = 300
    o = rng.uniform(-0.6, 0.6, (n, 3)).astype(np.float32)
    w = rng.normal(size=(n, 3))
    w = (w / np.linalg.norm(w, axis=1, keepdims=True)).astype(np.float32)
    dgt = rng.uniform(0.0, 0.8, n)
    hit = (rng.random(n) < 0.6).astype(np.uint8)
    shapes = [(Wd, E)] + [(Wd, Wd)] * (L - 1)
    hidden = [(rng.normal(size=s) / np.sqrt(s[1]), rng.uniform(-0.1, 0.1, s[0])) for s in shapes]
    head = (rng.normal(size=(2, Wd)) / np.sqrt(Wd), np.array([0.3, 0.0]))
    # torch model
    layers = []
    for W_, b_ in hidden:
        lin = torch.nn.Linear(W_.shape[1], W_.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W_))
            lin.bias.copy_(torch.from_numpy(b_))
        layers.append(torch.nn.utils.parametrizations.weight_norm(lin, dim=0))
    out = torch.nn.Linear(Wd, 1).double()
    with torch.no_grad():
        out.weight.copy_(torch.from_numpy(head[0][:1]))
        out.bias.copy_(torch.from_numpy(head[1][:1]))
    X, _ = omlp.encode(o, w, F)
    a = torch.from_numpy(X)
    for lin in layers:
        a = torch.relu(lin(a))
    yt = out(a)[:, 0]
    tgt = _torch_target(dgt, hit)
    if loss == "clamp":
        Lt = torch.mean(torch.abs(torch.clamp(tgt, -delta, delta) - torch.clamp(yt, -delta, delta)))
    else:
        Lt = torch.mean(torch.abs(torch.tanh(tgt) - torch.tanh(yt)))
    Lt.backward()
    # oracle composition
    vg = [H.wn_init(W_) for W_, _ in hidden]
    params = H.derive_single_head([(H.wn_fold(v, g), b_) for (v, g), (_, b_) in zip(vg, hidden)] + [head], delta)
    y, pres, acts = omlp.forward(params, X)
    if loss == "clamp":
        L64, gy = H.clamp_loss_and_output_grad(y, dgt, hit, delta)
    else:
        L64, gy = H.squish_loss_and_output_grad(y, dgt, hit)
    grads, _ = omlp.backward(params, pres, acts, gy)
    assert abs(L64 - Lt.item()) < 1e-12
    for (v, g), (dW, db), lin in zip(vg, grads[:-1], layers):
        dv, dg = H.wn_grad(v, g, dW)
        pw = lin.parametrizations.weight
        assert np.allclose(dv, pw.original1.grad.numpy(), rtol=1e-9, atol=1e-14)
        assert np.allclose(dg, pw.original0.grad.numpy()[:, 0], rtol=1e-9, atol=1e-14)
        assert np.allclose(db, lin.bias.grad.numpy(), rtol=1e-9, atol=1e-14)
    dWo, dbo = grads[-1]
    assert np.allclose(dWo[0], out.weight.grad.numpy()[0], rtol=1e-9, atol=1e-14)
    assert np.allclose(dbo[0], out.bias.grad.numpy()[0], rtol=1e-9, atol=1e-14)
    assert (dWo[1] == 0).all() and dbo[1] == 0
