"""Checkpoint / resume and the training forward pass: a handle saved after one Adam step and
loaded back continues bit-identically to the original (weights, moments and step count are all
restored), for the FP32 and the BF16 tensor-core training paths; ddf_forward_train returns the
query's distance and logit."""

import numpy as np
import pytest
import torch

from ddf_synth import init_weights
from oracle.sphere import sphere_ddf
from tests._helpers import ensure_built, rays_in_ball

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


def _batch(n, seed):
    o, w = rays_in_ball(n, seed=seed)
    dist, hit, _ = sphere_ddf(o, w, 0.5)
    dgt = np.where(hit, dist, np.inf).astype(np.float32)
    return [torch.from_numpy(x).cuda() for x in (o, w, dgt, hit.astype(np.uint8))]


@pytest.mark.parametrize("precision,shape", [("fp32", (12, 64, 3)), ("bf16", (12, 256, 4)),
                                             ("bf16", (0, 128, 2))])
def test_save_load_resumes_bit_identically(P, tmp_path, precision, shape):
    F, W, L = shape
    net = P.DDFNet(F, W, L, init_weights(F, W, L, seed=3), precision)
    b1, b2 = _batch(3000, 1), _batch(3000, 2)
    net.train_step(*b1, lr=1e-3)
    path = tmp_path / "net.ckpt"
    net.save(path)
    back = P.DDFNet.load(path)
    assert back.n_params == net.n_params
    assert torch.equal(back.get_weights(), net.get_weights())
    l_a = net.train_step(*b2, lr=1e-3)
    l_b = back.train_step(*b2, lr=1e-3)
    net.device_status()
    back.device_status()
    assert torch.equal(l_a, l_b)
    assert torch.equal(back.get_weights(), net.get_weights())    # Adam moments and step restored
    o, w = b1[0], b1[1]
    qa, qb = net.query(o, w), back.query(o, w)
    assert torch.equal(qa["dist"], qb["dist"])                    # same precision restored


def test_forward_train_matches_query(P):
    F, W, L = 12, 256, 4
    for precision in ("fp32", "bf16"):
        net = P.DDFNet(F, W, L, init_weights(F, W, L, seed=5), precision)
        o, w = [torch.from_numpy(x).cuda() for x in rays_in_ball(5000, seed=9)]
        d, z = net.forward_train(o, w)
        q = net.query(o, w)
        assert torch.equal(d, q["dist"]) and torch.equal(z, q["logit"])
