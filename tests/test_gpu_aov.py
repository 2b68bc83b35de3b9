"""AOV renders (the t-value and normal images of Fig. 3 / Fig. 4) on the GPU against the FP64
oracle (oracle/render.py, pinned to closed forms): the analytic sphere field, an FP32 network
(against the FP64 network) and a BF16 one (against the numpy model of its rounding points), and
the same pixel rays cast against a mesh by the labeller."""

import numpy as np
import pytest
import torch

from ddf_synth import default_camera, icosphere, torus_knot
from oracle import mlp as omlp
from oracle.mlp import normal_from_gradient
from oracle.render import field_aov, mesh_aov, primary_rays
from oracle.sphere import sphere_ddf
from tests._bf16_model import query_bf16
from tests._helpers import LOGIT_MARGIN, NETS, ensure_built, net_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


def _np(t):
    return t.cpu().numpy().reshape(t.shape[0] * t.shape[1], -1).squeeze()


def test_sphere_field_aov(P):
    cam = default_camera(96, 80, seed=2)
    r = 0.45
    depth, normal = P.DDFNet.sphere(r).render_aov(cam)
    gd, gn = _np(depth), _np(normal)

    def q(o, w):
        d, hit, g = sphere_ddf(o, w, r)
        return {"dist": np.where(hit, d, 0.0), "logit": np.where(hit, 1.0, -1.0), "normal": normal_from_gradient(g, w)}
    rd, rn, _ = field_aov(q, cam)
    # leave out rays within rounding of tangency
    _, w, _ = primary_rays(cam, np.arange(96 * 80), 1)
    e = np.array(cam.eye)
    b = w @ e
    clear = np.abs(b * b - (e @ e - r * r)) > 1e-4
    assert clear.mean() > 0.97
    hit = np.isfinite(rd)
    assert np.array_equal(np.isfinite(gd)[clear], hit[clear]) and 0.2 < hit.mean() < 0.8
    h = clear & hit
    assert np.abs(gd[h] - rd[h]).max() < 1e-5
    assert np.abs(gn[h] - rn[h]).max() < 1e-3
    assert (gn[~np.isfinite(gd)] == 0).all()


# the GPU's camera rays are float32 and differ from the oracle's by rounding; at BF16 that moves an
# encoded feature across a BF16 rounding boundary now and then (~1e-3 in the outputs), hence the
# wider BF16 margin and tolerance
@pytest.mark.parametrize("precision,tol,decide", [("fp32", 1e-4, LOGIT_MARGIN), ("bf16", 5e-3, 5e-3)])
def test_network_field_aov(P, precision, tol, decide):
    name = "train_78x256x8"
    F, W, L, _, _ = NETS[name]
    cam = default_camera(64, 48, seed=4)
    # shift the logit bias so that about half the pixels miss
    blob = net_weights(name)
    o, w, alive = primary_rays(cam, np.arange(64 * 48), 1)
    z = omlp.query(omlp.unpack(blob, F, W, L), o[alive], w[alive], F)["logit"]
    blob[-1] -= np.float32(np.median(z))
    net = P.DDFNet(F, W, L, blob, precision)
    depth, normal = net.render_aov(cam)
    gd, gn = _np(depth), _np(normal)
    Pm = omlp.unpack(blob, F, W, L)
    # the BF16 path against the numpy model of its rounding points
    qf = (lambda o, w: omlp.query(Pm, o, w, F)) if precision == "fp32" else (lambda o, w: query_bf16(Pm, o, w, F))
    rd, rn, margin = field_aov(qf, cam)
    ok = margin > decide
    print(f"{precision}: {ok.mean():.4f} of pixels clear of the hit threshold, {np.isfinite(rd).mean():.3f} hit")
    assert ok.mean() > 0.75 and 0.3 < np.isfinite(rd).mean() < 0.7
    assert np.array_equal(np.isfinite(gd)[ok], np.isfinite(rd)[ok])
    h = ok & np.isfinite(rd)
    assert h.sum() > 100
    assert np.abs(gd[h] - rd[h]).max() <= tol * max(1.0, np.abs(rd[h]).max())
    cos = np.sum(gn[h] * rn[h], 1)
    # (BF16: a perturbed input can also flip a ReLU mask, which moves the gradient)
    assert np.quantile(cos, 0.01) > (0.999 if precision == "fp32" else 0.95) and np.median(cos) > 0.9999


@pytest.mark.parametrize("mesh", ["icosphere", "knot"])
def test_mesh_aov(P, mesh):
    V, T = icosphere(2, 0.5) if mesh == "icosphere" else torus_knot(3, 2, 0.08, 64, 8)
    cam = default_camera(64, 56, seed=6)
    depth, normal, tri = P.DDFMesh(V, T).render_aov(cam)
    gd, gn, gt = _np(depth), _np(normal), _np(tri)
    # the GPU's float32 camera rays differ from the oracle's by rounding: compare the hit face,
    # and depth and normal where it agrees
    rd, rn, rt, _, w = mesh_aov(V, T, cam)
    same = gt == rt
    print(f"{mesh}: face agrees on {same.mean():.5f} of pixels; {(rt >= 0).mean():.3f} hit")
    assert same.mean() > 0.995
    h = same & (rt >= 0)
    assert np.abs(gd[h] - rd[h]).max() <= 1e-5 * max(1.0, rd[h].max())
    assert np.abs(gn[h] - rn[h]).max() < 1e-5
    assert np.isinf(gd[gt < 0]).all() and (gn[gt < 0] == 0).all()
