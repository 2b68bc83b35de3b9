"""GPU FP8 E4M3 query path (per-output-channel weight scales, static per-input-channel
activation scales from a calibration pass): against a model of its quantisation given the
library's scales (tests/_fp8_model.py) and, with the error stated, against the FP64 oracle; the
scales against their definition; FP8 renders run with Eq. 3 normals from the BF16 reverse pass."""

import numpy as np
import pytest
import torch

from ddf_synth import default_camera, init_weights
from oracle import mlp as omlp
from tests._fp8_model import calibration_bound, query_fp8
from tests._helpers import ensure_built, rays_in_ball

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


@pytest.mark.parametrize("F,W,L,seed", [(12, 256, 8, 2), (12, 128, 4, 7), (16, 256, 5, 4), (0, 128, 6, 9),
                                        (16, 512, 8, 5), (16, 512, 3, 6)])
@pytest.mark.parametrize("n", [1, 129, 4000])
def test_fp8_query_against_model_and_oracle(P, F, W, L, seed, n):
    blob = init_weights(F, W, L, seed=seed)
    net = P.DDFNet(F, W, L, blob, "fp8")
    o, w = rays_in_ball(n, seed=3 * n + W)
    out = net.query(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda(), normals=True)
    net.device_status()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    Pm = omlp.unpack(blob, F, W, L)
    m = query_fp8(Pm, o, w, F, net.fp8_scales())
    d = np.abs(g["dist"] - m["dist"])
    assert np.quantile(d, 0.99) <= 5e-3 and d.max() <= 3e-2, (np.quantile(d, 0.99), d.max())
    clear = np.abs(m["logit"]) >= 0.05
    assert (g["hit"][clear] == m["hit"][clear]).all()
    r = omlp.query(Pm, o, w, F, with_normal=False)
    err = np.abs(g["dist"] - r["dist"])
    print(f"FP8 {F},{W},{L}: |d dist| vs FP64 max {err.max():.4f} p99 {np.quantile(err, 0.99):.4f}")
    assert err.max() <= 0.2
    hit = g["hit"] == 1
    if hit.any():
        assert np.allclose(np.linalg.norm(g["normal"][hit], axis=1), 1.0, atol=1e-5)


def test_fp8_render_runs_and_tracks_bf16(P):
    F, W, L, seed = 12, 256, 8, 2
    blob = init_weights(F, W, L, seed=seed)
    n8 = P.DDFNet(F, W, L, blob, "fp8")
    n16 = P.DDFNet(F, W, L, blob, "bf16")
    cam = default_camera(32, 32)
    a = n8.render(cam, 4, 3).cpu().numpy()
    b = n16.render(cam, 4, 3).cpu().numpy()
    n8.device_status()
    assert np.isfinite(a).all()
    print(f"FP8 vs BF16 render mean |d pixel| = {np.abs(a - b).mean():.4f}")
    assert np.abs(a - b).mean() < 0.1


def _calibration_rays(n=8192, seed=0x43414C4942):
    """The library's calibration rays, rebuilt from their stated definition: Philox4x32-10 with
    key = seed, counter (i, 0, 0, 0) gives the origin (z = 1 - 2 u0, phi = 2 pi u1, r = cbrt(u2),
    uniform in the unit ball) and counter (i, 0, 1, 0) the direction (z = 1 - 2 u0, phi = 2 pi u1)."""
    from oracle.philox import path_uniforms
    ids = np.arange(n)
    a = path_uniforms(seed, ids, 0)
    b = path_uniforms(seed, ids, 1)
    z0, p0, r0 = 1 - 2 * a[:, 0], 2 * np.pi * a[:, 1], np.cbrt(a[:, 2])
    s0 = np.sqrt(np.maximum(0, 1 - z0 * z0))
    o = np.stack([r0 * s0 * np.cos(p0), r0 * s0 * np.sin(p0), r0 * z0], 1)
    z1, p1 = 1 - 2 * b[:, 0], 2 * np.pi * b[:, 1]
    s1 = np.sqrt(np.maximum(0, 1 - z1 * z1))
    w = np.stack([s1 * np.cos(p1), s1 * np.sin(p1), z1], 1)
    return o.astype(np.float32), w.astype(np.float32)


@pytest.mark.parametrize("F,W,L,seed", [(12, 256, 8, 2), (0, 128, 6, 9), (16, 512, 8, 5)])
def test_fp8_static_scales_cover_the_activations(P, F, W, L, seed):
    """Layer 0's scale is 1/448; a hidden layer's is twice the channel's calibration maximum
    (floored at 1e-3 of the layer's maximum) / 448: compared with the FP64 column maxima on the
    same 8,192 calibration rays (the library's maxima come from its BF16 forward)."""
    blob = init_weights(F, W, L, seed=seed)
    net = P.DDFNet(F, W, L, blob, "fp8")
    sa = net.fp8_scales().astype(np.float64)
    assert (sa[0] == np.float32(1 / 448)).all()
    o, w = _calibration_rays()
    c = calibration_bound(omlp.unpack(blob, F, W, L), o, w, F)
    for l in range(1, L):
        g = sa[l] * 448 / 2
        assert (g >= 1e-3 * g.max() * (1 - 1e-6)).all()
        live = c[l] > 0.05 * c[l].max()
        ratio = g[live] / c[l][live]
        assert 0.95 <= ratio.min() and ratio.max() <= 1.05, (l, ratio.min(), ratio.max())


def test_fp8_scales_follow_set_weights(P):
    """Repacking after new weights recalibrates: doubling every weight of layer 0 doubles the
    activations of layer 1 and so its scales (to BF16 rounding)."""
    F, W, L, seed = 12, 128, 4, 5
    blob = init_weights(F, W, L, seed=seed)
    net = P.DDFNet(F, W, L, blob, "fp8")
    s1 = net.fp8_scales()
    Pm = omlp.unpack(blob, F, W, L)
    blob2 = blob.copy()
    n0 = Pm[0][0].size + Pm[0][1].size
    blob2[:n0] *= 2
    net.set_weights(torch.from_numpy(blob2).cuda())
    s2 = net.fp8_scales()
    assert (s2[0] == s1[0]).all()
    r = s2[1] / s1[1]
    assert np.allclose(r, 2.0, rtol=2e-2), (r.min(), r.max())


def test_fp8_width512_full_size_sampled(P):
    """2^22 queries of the 102 -> 512 x 8 -> 2 network in one FP8 launch (the large-render shape):
    2,000 sampled rows against the quantisation model and, with the error stated, the FP64 oracle;
    normals (from the BF16 reverse pass) are unit vectors on the hit rows."""
    F, W, L, seed = 16, 512, 8, 5
    blob = init_weights(F, W, L, seed=seed)
    net = P.DDFNet(F, W, L, blob, "fp8")
    n = 1 << 22
    g = torch.Generator(device="cuda").manual_seed(8)
    o = torch.randn(n, 3, device="cuda", generator=g)
    o = o / o.norm(dim=1, keepdim=True) * torch.rand(n, 1, device="cuda", generator=g)
    w = torch.randn(n, 3, device="cuda", generator=g)
    w = w / w.norm(dim=1, keepdim=True)
    out = net.query(o, w, normals=True)
    net.device_status()
    idx = np.random.default_rng(1).choice(n, 2000, replace=False)
    idx[:2] = [0, n - 1]
    on, wn = o[idx].cpu().numpy(), w[idx].cpu().numpy()
    gs = {k: v[idx].cpu().numpy() for k, v in out.items()}
    Pm = omlp.unpack(blob, F, W, L)
    m = query_fp8(Pm, on, wn, F, net.fp8_scales())
    d = np.abs(gs["dist"] - m["dist"])
    assert np.quantile(d, 0.99) <= 5e-3 and d.max() <= 3e-2, (np.quantile(d, 0.99), d.max())
    clear = np.abs(m["logit"]) >= 0.05
    assert (gs["hit"][clear] == m["hit"][clear]).all()
    r = omlp.query(Pm, on, wn, F, with_normal=False)
    err = np.abs(gs["dist"] - r["dist"])
    print(f"FP8 102 -> 512 x 8 at 2^22 rows: |d dist| vs FP64 max {err.max():.4f} p99 {np.quantile(err, 0.99):.4f}")
    assert err.max() <= 0.2
    hit = gs["hit"] == 1
    if hit.any():
        assert np.allclose(np.linalg.norm(gs["normal"][hit], axis=1), 1.0, atol=1e-5)
    # the same rows through the BF16 handle: both tensor-core paths agree with each other loosely
    net.set_precision("bf16")
    b = net.query(o, w)
    diff = (b["dist"][torch.from_numpy(idx).cuda()].cpu().numpy() - gs["dist"])
    assert np.abs(diff).max() <= 0.2
