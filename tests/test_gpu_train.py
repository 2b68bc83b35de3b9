"""GPU reverse pass and training step against the FP64 oracle gradient (which is itself pinned
to finite differences and torch autograd): per-tensor relative L2 error of the weight and input
gradients, determinism, the recompute path and the Adam step."""

import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from tests._helpers import NETS, ensure_built, net_weights, rays_in_ball

pytestmark = pytest.mark.gpu

GRAD_REL = 1e-4


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _blob_split(blob, name):
    F, W, L, _, _ = NETS[name]
    return omlp.unpack(blob, F, W, L)


@pytest.mark.parametrize("name,n", [("tiny_6x64x4", 1000), ("train_78x256x8", 1024)])
def test_backward_matches_oracle(P, name, n):
    F, W, L, _, _ = NETS[name]
    o, w = rays_in_ball(n, seed=21)
    rng = np.random.default_rng(3)
    gd = rng.normal(size=n).astype(np.float32)
    gl = rng.normal(size=n).astype(np.float32)
    net = P.DDFNet(F, W, L, net_weights(name))
    to, tw = torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()
    gw, gin = net.backward(to, tw, torch.from_numpy(gd).cuda(), torch.from_numpy(gl).cuda(), need_input=True)
    gw2, _ = net.backward(to, tw, torch.from_numpy(gd).cuda(), torch.from_numpy(gl).cuda())
    torch.cuda.synchronize()
    assert torch.equal(gw, gw2)                                      # deterministic
    Pm = _blob_split(net_weights(name), name)
    X, dX = omlp.encode(o, w, F)
    y, pres, acts = omlp.forward(Pm, X)
    grads, gX = omlp.backward(Pm, pres, acts, np.stack([gd, gl], 1).astype(np.float64))
    ref = omlp.pack(grads)
    got = gw.cpu().numpy().astype(np.float64)
    for (dW, db), (gW, gb) in zip(grads, _blob_split(got, name)):
        assert _rel(gW, dW) < GRAD_REL
        assert _rel(gb, db) < GRAD_REL
    gi = np.zeros((n, 6))
    gf = gX * dX
    for f in range(X.shape[1]):
        gi[:, f % 6] += gf[:, f]
    assert _rel(gin.cpu().numpy(), gi) < GRAD_REL
    assert ref.size == got.size


def test_backward_recompute_chunks(P):
    """A small workspace cap forces many row chunks; the gradient stays within FP32 rounding."""
    name = "train_78x256x8"
    F, W, L, _, _ = NETS[name]
    n = 3000
    o, w = rays_in_ball(n, seed=5)
    net = P.DDFNet(F, W, L, net_weights(name))
    to, tw = torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()
    gd = torch.ones(n, device="cuda")
    gl = torch.full((n,), -0.5, device="cuda")
    full, _ = net.backward(to, tw, gd, gl)
    net.set_workspace_limit(1 << 20)        # ~ 256-row chunks
    chunked, _ = net.backward(to, tw, gd, gl)
    torch.cuda.synchronize()
    a, b = chunked.cpu().numpy(), full.cpu().numpy()
    assert _rel(a, b) < 1e-5


def test_autograd_function(P):
    name = "tiny_6x64x4"
    F, W, L, _, _ = NETS[name]
    n = 512
    o, w = rays_in_ball(n, seed=8)
    net = P.DDFNet(F, W, L, net_weights(name))
    weights = torch.from_numpy(net_weights(name)).cuda().requires_grad_(True)
    to = torch.from_numpy(o).cuda().requires_grad_(True)
    tw = torch.from_numpy(w).cuda()
    dist, logit, hit = P.ddf_apply(net, weights, to, tw)
    loss = (dist * 2.0).sum() + logit.sum()
    loss.backward()
    Pm = _blob_split(net_weights(name), name)
    X, dX = omlp.encode(o, w, F)
    y, pres, acts = omlp.forward(Pm, X)
    gy = np.stack([np.full(n, 2.0), np.ones(n)], 1)
    grads, gX = omlp.backward(Pm, pres, acts, gy)
    assert _rel(weights.grad.cpu().numpy(), omlp.pack(grads)) < GRAD_REL
    gi = np.zeros((n, 6))
    gf = gX * dX
    for f in range(X.shape[1]):
        gi[:, f % 6] += gf[:, f]
    assert _rel(to.grad.cpu().numpy(), gi[:, :3]) < GRAD_REL


def test_train_step_loss_and_update(P):
    name = "train_78x256x8"
    F, W, L, _, _ = NETS[name]
    n = 2048
    o, w = rays_in_ball(n, seed=12)
    rng = np.random.default_rng(2)
    dgt = rng.uniform(0, 1.5, n).astype(np.float32)
    hgt = (rng.random(n) < 0.5).astype(np.uint8)
    dgt[hgt == 0] = np.inf
    blob = net_weights(name)
    net = P.DDFNet(F, W, L, blob)
    loss = net.train_step(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda(),
                          torch.from_numpy(dgt).cuda(), torch.from_numpy(hgt).cuda(), lr=1e-3)
    new = net.get_weights().cpu().numpy().astype(np.float64)
    Pm = _blob_split(blob, name)
    L64, grads, _ = omlp.param_gradient(Pm, o, w, F, dgt, hgt)
    assert abs(loss.item() - L64) <= 1e-5 * max(1.0, abs(L64))
    g = omlp.pack(grads)
    w1, _, _ = omlp.adam_update(blob.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1,
                                1e-3, 0.9, 0.999, 1e-8)
    # at step 1 Adam moves each weight by ~lr * sign(g); compare where |g| is clearly non-zero
    big = np.abs(g) > 1e-4 * np.abs(g).max()
    assert big.mean() > 0.5
    assert np.allclose(new[big], w1[big], rtol=0, atol=2e-6)
    assert np.all(np.abs(new - blob) <= 1e-3 * 1.0001 + 1e-7)
