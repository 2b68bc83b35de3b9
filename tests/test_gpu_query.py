"""GPU parity of the batched DDF query (distance, logit, hit, Eq. 3 normal) against the FP64
oracle, element by element, through the C ABI."""

import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from oracle.sphere import sphere_ddf
from tests._helpers import (LOGIT_MARGIN, NETS, ensure_built, fp32_close, net_weights, rays_in_ball)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


def _oracle(name, o, w, normals=True):
    F, W, L, _, _ = NETS[name]
    P = omlp.unpack(net_weights(name), F, W, L)
    return omlp.query(P, o, w, F, with_normal=normals)


def _gpu(lib, name, o, w, normals=True, precision="fp32"):
    F, W, L, _, _ = NETS[name]
    net = lib.DDFNet(F, W, L, net_weights(name), precision)
    out = net.query(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda(), normals=normals)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def _check_fp32(g, r, normals=True):
    assert fp32_close(g["dist"], r["dist"]).all(), np.max(np.abs(g["dist"] - r["dist"]))
    assert fp32_close(g["logit"], r["logit"]).all(), np.max(np.abs(g["logit"] - r["logit"]))
    clear = np.abs(r["logit"]) >= LOGIT_MARGIN
    assert (g["hit"][clear] == r["hit"][clear]).all()
    if normals:
        h = (g["hit"] == 1) & clear
        gn = np.linalg.norm(r["grad"][:, :3], axis=1)
        ok = h & (gn > 1e-3)
        assert np.allclose(g["normal"][ok], r["normal"][ok], atol=1e-4)
        assert (g["normal"][g["hit"] == 0] == 0).all()    # only hit rows are written


@pytest.mark.parametrize("name", list(NETS))
@pytest.mark.parametrize("n", [1, 63, 1000, 4097])
def test_fp32_query_parity(lib, name, n):
    o, w = rays_in_ball(n, seed=100 + n)
    _check_fp32(_gpu(lib, name, o, w), _oracle(name, o, w))


def test_fp32_query_deep_network(lib):
    """16 hidden layers at width 256: the FP32 kernel's shared memory then holds one weight-chunk
    buffer instead of two (the chunks are copied and multiplied in turn); same parity."""
    from ddf_synth import init_weights
    F, W, L = 12, 256, 16
    blob = init_weights(F, W, L, seed=6)
    o, w = rays_in_ball(1000, seed=61)
    net = lib.DDFNet(F, W, L, blob, "fp32")
    out = net.query(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda(), normals=True)
    torch.cuda.synchronize()
    g = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    _check_fp32(g, omlp.query(omlp.unpack(blob, F, W, L), o, w, F, with_normal=True))


def test_fp32_query_empty(lib):
    F, W, L, _, _ = NETS["tiny_6x64x4"]
    net = lib.DDFNet(F, W, L, net_weights("tiny_6x64x4"))
    z = torch.empty(0, 3, device="cuda")
    out = net.query(z, z, normals=True)
    assert out["dist"].numel() == 0


def test_fp32_query_full_size_sampled(lib):
    """2^24 queries of the 78 -> 256 x 8 network in one launch; 2,000 sampled rows checked."""
    name = "train_78x256x8"
    n = 1 << 24
    g = torch.Generator(device="cuda").manual_seed(7)
    o = torch.randn(n, 3, device="cuda", generator=g)
    o = o / o.norm(dim=1, keepdim=True) * torch.rand(n, 1, device="cuda", generator=g)
    w = torch.randn(n, 3, device="cuda", generator=g)
    w = w / w.norm(dim=1, keepdim=True)
    F, W, L, _, _ = NETS[name]
    net = lib.DDFNet(F, W, L, net_weights(name))
    out = net.query(o, w, normals=True)
    torch.cuda.synchronize()
    idx = np.random.default_rng(0).choice(n, 2000, replace=False)
    idx[:2] = [0, n - 1]
    on, wn = o[idx].cpu().numpy(), w[idx].cpu().numpy()
    gsub = {k: v[idx].cpu().numpy() for k, v in out.items()}
    _check_fp32(gsub, _oracle(name, on, wn))


def test_sphere_field_query(lib):
    o, w = rays_in_ball(3000, seed=4)
    o = o / np.linalg.norm(o, axis=1, keepdims=True).astype(np.float32)
    net = lib.DDFNet.sphere(0.5)
    out = net.query(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda(), normals=True)
    torch.cuda.synchronize()
    d, h, gr = sphere_ddf(o, w, 0.5)
    disc_margin = np.abs(np.sum(o * w, 1) ** 2 - (np.sum(o * o, 1) - 0.25)) > 1e-5
    hh = out["hit"].cpu().numpy().astype(bool)
    assert (hh[disc_margin] == h[disc_margin]).all()
    both = hh & h & disc_margin
    assert np.allclose(out["dist"].cpu().numpy()[both], d[both], rtol=1e-5, atol=1e-6)
    nrm = omlp.normal_from_gradient(gr, w)
    assert np.allclose(out["normal"].cpu().numpy()[both], nrm[both], atol=1e-4)
