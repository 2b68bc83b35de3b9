"""The GPU FP32 reverse pass (ddf_backward) against FP64 central finite differences of the
network itself, with no analytic gradient in between: on 1,024 rays of the training set (origins
on the bounding sphere, half aimed at the (3,2) knot's surface, labelled against its 8,192 faces)
and the training network 78 -> 256 x 8 -> 2 (Sec. 5.1's setting with this build's encoding).

The cotangents are the loss's dLoss/dy at the current weights (L1 on labelled hits + BCE, rounded
to float32 once), so the GPU returns the training gradient. The finite differences are of
Phi(W) = sum_i c_i . y_i(W) in float64 with those cotangents held fixed, whose gradient the GPU
gradient is: along 16 random directions of the whole weight vector, along 256 single weights
and biases, and for all six ray coordinates of every ray. A step whose +-h passes change a ReLU
mask is shrunk (a kink would make the difference meaningless); a ray coordinate whose passes
change a mask of that ray is left out and counted."""

import numpy as np
import pytest
import torch

from ddf_synth import init_weights, labelled_ray_set, torus_knot
from oracle import mlp as omlp
from oracle.label import label_rays

pytestmark = pytest.mark.gpu

F, W, L, SEED = 12, 256, 8, 2


@pytest.fixture(scope="module")
def setup():
    from tests._helpers import ensure_built
    ensure_built()
    import paper_2306_16142_gb300 as P
    V, T = torus_knot(3, 2, 0.08, 256, 16)
    o, w = labelled_ray_set(V, T, 1024, seed=31)
    d, h, _, _ = label_rays(V, T, o, w)
    blob = init_weights(F, W, L, seed=SEED)
    Pm = omlp.unpack(blob, F, W, L)
    X, _ = omlp.encode(o, w, F)
    y, _, _ = omlp.forward(Pm, X)
    _, gy = omlp.loss_and_output_grad(y, np.where(h == 1, d, np.inf), h)
    c = gy.astype(np.float32)
    net = P.DDFNet(F, W, L, blob, "fp32")
    gw, gin = net.backward(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda(),
                           torch.from_numpy(np.ascontiguousarray(c[:, 0])).cuda(),
                           torch.from_numpy(np.ascontiguousarray(c[:, 1])).cuda(), need_input=True)
    torch.cuda.synchronize()
    return dict(o=o, w=w, blob=blob.astype(np.float64), c=c.astype(np.float64),
                gw=gw.cpu().numpy().astype(np.float64), gin=gin.cpu().numpy().astype(np.float64),
                hits=int(h.sum()))


def _phi(blob, X, c):
    """Per-ray c_i . y_i and the ReLU masks, in float64."""
    y, pres, _ = omlp.forward(omlp.unpack(blob, F, W, L), X)
    return np.sum(c * y, axis=1), [z > 0 for z in pres]


def _same_masks(ma, mb):
    return all(np.array_equal(a, b) for a, b in zip(ma, mb))


def _fd_direction(blob, X, c, v, h0):
    h = h0
    for _ in range(4):
        pa, ma = _phi(blob + h * v, X, c)
        pb, mb = _phi(blob - h * v, X, c)
        if _same_masks(ma, mb):
            return (np.sum(pa) - np.sum(pb)) / (2 * h)
        h /= 10
    pytest.fail("every step crossed a ReLU kink")


def test_weight_gradient_against_central_differences(setup):
    s = setup
    assert s["hits"] > 50
    X, _ = omlp.encode(s["o"], s["w"], F)
    rng = np.random.default_rng(5)
    gnorm = np.linalg.norm(s["gw"])
    worst = 0.0
    for _ in range(16):
        v = rng.normal(size=s["blob"].size)
        v /= np.linalg.norm(v)
        fd = _fd_direction(s["blob"], X, s["c"], v, 1e-6)
        got = float(s["gw"] @ v)
        err = abs(got - fd) / (abs(fd) + 1e-3 * gnorm)
        worst = max(worst, err)
        assert err <= 1e-4, (got, fd)
    idx = rng.choice(s["blob"].size, 256, replace=False)
    for k in idx:
        v = np.zeros(s["blob"].size)
        v[k] = 1.0
        fd = _fd_direction(s["blob"], X, s["c"], v, 1e-6)
        assert abs(s["gw"][k] - fd) <= 1e-4 * abs(fd) + 1e-6 * gnorm, (k, s["gw"][k], fd)
    print(f"weight gradient vs FP64 central differences: worst relative error {worst:.2e} over 16 directions")


def test_input_gradient_against_central_differences(setup):
    s = setup
    o, w, c = s["o"].astype(np.float64), s["w"].astype(np.float64), s["c"]
    h = 1e-7
    skipped = 0
    scale = np.max(np.abs(s["gin"]))
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        oa, wa = o + e[None, :3], w + e[None, 3:]
        ob, wb = o - e[None, :3], w - e[None, 3:]
        pa, ma = _phi(s["blob"], omlp.encode(oa, wa, F)[0], c)
        pb, mb = _phi(s["blob"], omlp.encode(ob, wb, F)[0], c)
        same = np.ones(o.shape[0], bool)
        for a, b in zip(ma, mb):
            same &= (a == b).all(axis=1)
        fd = (pa - pb) / (2 * h)
        got = s["gin"][:, j]
        err = np.abs(got - fd)
        assert (err[same] <= 1e-4 * np.abs(fd[same]) + 1e-6 * scale).all(), err[same].max()
        skipped += int((~same).sum())
    assert skipped <= 6 * 1024 // 50
    print(f"input gradient vs FP64 central differences: {6 * 1024 - skipped} ray coordinates, {skipped} at a kink")
