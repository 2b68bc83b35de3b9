"""GPU FP8 E4M3 query path (per-output-channel weight scales, per-row activation scales):
against a model of its quantisation (tests/_fp8_model.py) and, with the error stated, against
the FP64 oracle; FP8 renders run with Eq. 3 normals from the BF16 reverse pass."""

import numpy as np
import pytest
import torch

from ddf_synth import default_camera, init_weights
from oracle import mlp as omlp
from tests._fp8_model import query_fp8
from tests._helpers import ensure_built, rays_in_ball

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


@pytest.mark.parametrize("F,W,L,seed", [(12, 256, 8, 2), (12, 128, 4, 7), (16, 256, 5, 4), (0, 128, 6, 9)])
@pytest.mark.parametrize("n", [1, 129, 4000])
def test_fp8_query_against_model_and_oracle(P, F, W, L, seed, n):
    blob = init_weights(F, W, L, seed=seed)
    net = P.DDFNet(F, W, L, blob, "fp8")
    o, w = rays_in_ball(n, seed=3 * n + W)
    out = net.query(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda(), normals=True)
    net.device_status()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    Pm = omlp.unpack(blob, F, W, L)
    m = query_fp8(Pm, o, w, F)
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
