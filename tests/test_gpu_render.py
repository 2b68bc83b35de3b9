"""GPU wavefront renderer against the FP64 path-tracer oracle: the convex closed form with the
analytic sphere field, and the FP32 network render per pixel (paths with a hit decision within
1e-4 of the threshold on the oracle side are exempt; their share is reported)."""

import numpy as np
import pytest
import torch

from ddf_synth import default_camera
from oracle import mlp as omlp
from oracle.render import mesh_query, primary_rays, render_pixels
from tests._helpers import LOGIT_MARGIN, NETS, ensure_built, net_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


@pytest.mark.parametrize("bounces,spp,size", [(3, 4, 32), (2, 7, 33)])
def test_sphere_closed_form_render(P, bounces, spp, size):
    cam = default_camera(size, size)
    net = P.DDFNet.sphere(0.5)
    img = net.render(cam, spp, bounces).cpu().numpy().ravel()
    pids = np.arange(size * size * spp)
    o, w, alive = primary_rays(cam, pids, spp)
    b = np.sum(o * w, 1)
    disc = b * b - (np.sum(o * o, 1) - 0.25)
    hitp = (disc >= 0) & (-b - np.sqrt(np.maximum(disc, 0)) > 0)
    k = hitp.reshape(-1, spp).sum(1)
    expect = (0.7 * k + (spp - k)) / spp
    clear = (np.abs(disc) > 1e-4).reshape(-1, spp).all(1)
    assert clear.mean() > 0.95
    assert np.allclose(img[clear], expect[clear], rtol=0, atol=2e-6)
    # every value is of the form (0.7 k + (spp - k)) / spp
    kk = np.round((1 - img) / 0.3 * spp)
    assert np.allclose(img, (0.7 * kk + (spp - kk)) / spp, atol=2e-6)
    stats = net.render_stats(bounces)
    assert stats[0] == size * size * spp


def test_fp32_network_render_parity(P):
    """The plain tiny configuration: 64 x 64 pixels, 4 spp, at most 3 bounces, 6 -> 64 x 4 -> 2."""
    name = "tiny_6x64x4"
    F, W, L, _, _ = NETS[name]
    cam = default_camera(64, 64)
    spp, bounces = 4, 3
    net = P.DDFNet(F, W, L, net_weights(name))
    img = net.render(cam, spp, bounces).cpu().numpy().ravel()
    img2 = net.render(cam, spp, bounces).cpu().numpy().ravel()
    assert (img.view(np.uint32) == img2.view(np.uint32)).all()       # order-independent, deterministic
    Pm = omlp.unpack(net_weights(name), F, W, L)
    ref = render_pixels(lambda o, w: omlp.query(Pm, o, w, F), cam, spp, bounces, np.arange(64 * 64))
    exempt_path = ref["min_abs_logit"] < LOGIT_MARGIN
    exempt_px = exempt_path.reshape(-1, spp).any(1)
    ok = ~exempt_px
    assert ok.mean() > 0.9, ok.mean()
    assert np.allclose(img[ok], ref["image"][ok], rtol=0, atol=1e-4)
    print(f"exempt paths {exempt_path.mean():.4%}, exempt pixels {exempt_px.mean():.4%}")
    # some paths bounce (not a trivially black or white image)
    assert 0.05 < np.mean(np.isclose(ref["radiance"], 0.7)) or np.mean(ref["radiance"] == 0) > 0.05


def test_render_spp1_per_path_parity(P):
    """With one sample per pixel every pixel is one path: compare every non-exempt path."""
    name = "tiny_6x64x4"
    F, W, L, _, _ = NETS[name]
    cam = default_camera(48, 40, seed=9)
    net = P.DDFNet(F, W, L, net_weights(name))
    img = net.render(cam, 1, 4).cpu().numpy().ravel()
    Pm = omlp.unpack(net_weights(name), F, W, L)
    ref = render_pixels(lambda o, w: omlp.query(Pm, o, w, F), cam, 1, 4, np.arange(48 * 40))
    ok = ref["min_abs_logit"] >= LOGIT_MARGIN
    assert np.allclose(img[ok], ref["image"][ok], rtol=0, atol=1e-6)


def test_mesh_render_convex_closed_form(P):
    """A convex mesh: a sample that meets it bounces away for good, so each pixel is
    (0.7 k + (spp - k)) / spp with k its samples that meet the mesh."""
    from ddf_synth import icosphere
    V, T = icosphere(3, 0.5)
    cam = default_camera(40, 40, seed=3)
    spp = 4
    img = P.DDFMesh(V, T).render(cam, spp, 3).cpu().numpy().ravel()
    kk = np.round((1 - img) / 0.3 * spp)
    assert np.allclose(img, (0.7 * kk + (spp - kk)) / spp, atol=2e-6)
    ref = render_pixels(mesh_query(V, T), cam, spp, 3, np.arange(40 * 40))
    same = np.abs(img - ref["image"]) < 1e-6
    print(f"convex mesh: {same.mean():.4f} of pixels equal the oracle")
    assert same.mean() > 0.97 and 0.1 < (kk > 0).mean() < 0.9


def test_mesh_render_two_spheres_against_the_oracle(P):
    """A non-convex scene (two spheres that light bounces between) against the oracle's path
    tracer driven by the FP64 labeller; pixels whose paths graze an edge may differ."""
    from ddf_synth import icosphere
    Va, Ta = icosphere(3, 0.3)
    V = np.concatenate([Va + np.float32([-0.35, 0, 0]), Va + np.float32([0.35, 0, 0])]).astype(np.float32)
    T = np.concatenate([Ta, Ta + Va.shape[0]]).astype(np.int32)
    cam = default_camera(32, 32, seed=5)
    spp, bounces = 4, 4
    mesh = P.DDFMesh(V, T)
    img = mesh.render(cam, spp, bounces).cpu().numpy().ravel()
    mesh.set_accel("none")
    img2 = mesh.render(cam, spp, bounces).cpu().numpy().ravel()
    assert np.array_equal(img, img2)                      # the same labels either way
    ref = render_pixels(mesh_query(V, T), cam, spp, bounces, np.arange(32 * 32))
    same = np.abs(img - ref["image"]) < 1e-6
    print(f"two spheres: {same.mean():.4f} of pixels equal the oracle, mean |diff| {np.abs(img - ref['image']).mean():.5f}")
    assert same.mean() > 0.9 and np.abs(img - ref["image"]).mean() < 0.02
    assert (ref["image"] < 0.7 - 1e-9).any()              # some paths do bounce between the spheres
