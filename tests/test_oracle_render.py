"""Pins of the FP64 path-tracer oracle and the analytic sphere DDF: the directed
Eikonal equation and t-shift (Eq. 2), the normal of Eq. 3, the orthonormal basis,
the moments of cosine-weighted sampling, the camera geometry and the convex closed
form of the render (every path that meets a convex Lambertian object returns exactly
the albedo, every other path the environment)."""

import math

import numpy as np
import pytest

from ddf_synth import default_camera
from oracle.philox import path_uniforms
from oracle.render import (camera_basis, cosine_direction, onb_duff, primary_rays,
                           render_pixels, trace_paths)
from oracle.sphere import sphere_ddf
from oracle.mlp import normal_from_gradient


def _rand_rays(n, seed):
    rng = np.random.default_rng(seed)
    o = rng.normal(size=(n, 3))
    o /= np.linalg.norm(o, axis=1, keepdims=True)
    w = -o + 0.4 * rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    return o, w


def test_sphere_eikonal_and_shift():
    o, w = _rand_rays(500, 1)
    d, hit, g = sphere_ddf(o, w, 0.5)
    assert hit.sum() > 100
    # Eq. 2: grad_x phi . theta = -1 on visible oriented points
    assert np.allclose(np.sum(g[hit] * w[hit], 1), -1.0, atol=1e-12)
    # phi(x) - phi(x + t theta) = t
    s = 0.3 * d[hit]
    d2, h2, _ = sphere_ddf(o[hit] + s[:, None] * w[hit], w[hit], 0.5)
    assert h2.all() and np.allclose(d[hit] - d2, s, atol=1e-12)
    # gradient against central differences
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        dp, _, _ = sphere_ddf(o[hit] + e, w[hit], 0.5)
        dm, _, _ = sphere_ddf(o[hit] - e, w[hit], 0.5)
        assert np.allclose((dp - dm) / (2 * h), g[hit, j], rtol=1e-5, atol=1e-6)
    # Eq. 3 gives the outward sphere normal at q
    q = o[hit] + d[hit, None] * w[hit]
    n = normal_from_gradient(g[hit], w[hit])
    assert np.allclose(n, q / 0.5, atol=1e-12)


def test_onb_duff_orthonormal():
    rng = np.random.default_rng(4)
    n = rng.normal(size=(2000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[0] = [0, 0, 1]
    n[1] = [0, 0, -1]
    b1, b2 = onb_duff(n)
    for a, b in [(b1, b2), (b1, n), (b2, n)]:
        assert np.allclose(np.sum(a * b, 1), 0, atol=1e-12)
    for a in (b1, b2):
        assert np.allclose(np.linalg.norm(a, axis=1), 1, atol=1e-12)
    assert np.allclose(np.cross(b1, b2), n, atol=1e-12)     # right-handed


def test_cosine_sampling_moments():
    rng = np.random.default_rng(8)
    N = 400000
    n = rng.normal(size=(N, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    u = path_uniforms(5, np.arange(N, dtype=np.uint64), 1)
    d = cosine_direction(n, u[:, 0], u[:, 1])
    c = np.sum(d * n, 1)
    assert (c >= 0).all() and np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-12)
    # cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2
    assert abs(c.mean() - 2 / 3) < 4 * math.sqrt(1 / 18 / N)
    assert abs((c * c).mean() - 0.5) < 4 * math.sqrt(1 / 12 / N)


def test_camera_geometry():
    cam = default_camera(64, 48)
    eye, f, r, u = camera_basis(cam)
    assert np.allclose(np.linalg.norm(eye), 2.5)
    assert np.allclose(f, -eye / 2.5)
    assert abs(r[2]) < 1e-15 and u[2] > 0
    pids = np.arange(64 * 48 * 2)
    o, w, alive = primary_rays(cam, pids, 2)
    # a ray meets the unit ball iff its angle to the eye->centre axis is below asin(1/2.5)
    ang_c = np.arccos(np.clip(w @ f, -1, 1))
    lim = math.asin(1 / 2.5)
    assert (alive[ang_c < lim - 1e-9]).all() and not alive[ang_c > lim + 1e-9].any()
    assert np.allclose(np.linalg.norm(o[alive], axis=1), 1.0, atol=1e-12)
    sq = default_camera(64, 64)
    assert primary_rays(sq, np.arange(64 * 64 * 2), 2)[2].all()   # square view: all rays meet it
    th = math.tan(math.radians(cam.vfov_deg / 2))
    half_diag = math.atan(th * math.hypot(1, 64 / 48))
    ang = np.arccos(np.clip(w @ f, -1, 1))
    assert ang.max() <= half_diag + 1e-12
    # pixel (0, 0) is at the top-left: up and left of the centre
    assert (w[0] @ u) > 0 and (w[0] @ r) < 0


def _sphere_query(r):
    def q(o, w):
        d, hit, g = sphere_ddf(o, w, r)
        n = normal_from_gradient(g, w)
        return {"dist": np.where(hit, d, 0.0), "logit": np.where(hit, 1.0, -1.0), "normal": n}
    return q


@pytest.mark.parametrize("bounces", [2, 3])
def test_convex_closed_form_render(bounces):
    cam = default_camera(32, 32)
    spp = 4
    pixels = np.arange(32 * 32)
    res = render_pixels(_sphere_query(0.5), cam, spp, bounces, pixels)
    # independent count of primary rays that meet the r = 0.5 sphere
    o, w, alive = primary_rays(cam, res["pids"], spp)
    b = np.sum(o * w, 1)
    disc = b * b - (np.sum(o * o, 1) - 0.25)
    k = ((disc >= 0) & (-b - np.sqrt(np.maximum(disc, 0)) > 0)).reshape(-1, spp).sum(1)
    expect = (0.7 * k + (spp - k)) / spp
    assert np.allclose(res["image"], expect, rtol=0, atol=1e-15)
    assert 0 < k.sum() < 32 * 32 * spp
    assert set(np.unique(res["radiance"]).tolist()) <= {0.7, 1.0}


def test_bounce_cap_gives_black():
    cam = default_camera(16, 16)
    res = render_pixels(_sphere_query(0.5), cam, 1, 1, np.arange(256))
    first_hit = res["logit"] > 0
    assert first_hit.any()
    assert (res["radiance"][first_hit] == 0).all() and (res["radiance"][~first_hit] == 1).all()


def test_mesh_tracer_convex_closed_form():
    """The path tracer with a convex mesh in place of the field (oracle.render.mesh_query): a
    sample that meets the mesh bounces away for good, so each pixel is (0.7 k + (spp - k)) / spp
    with k its primary rays that meet the mesh, counted here by an independent ray-sphere
    bracket: rays missing the circumscribed sphere miss, rays meeting the inscribed one hit."""
    from ddf_synth import icosphere
    from oracle.render import mesh_query
    V, T = icosphere(2, 0.5)
    cam = default_camera(24, 24, seed=2)
    spp = 4
    res = render_pixels(mesh_query(V, T), cam, spp, 3, np.arange(24 * 24))
    kk = np.round((1 - res["image"]) / 0.3 * spp)
    assert np.allclose(res["image"], (0.7 * kk + (spp - kk)) / spp, atol=1e-12)
    o, w, alive = primary_rays(cam, res["pids"], spp)
    b = np.sum(o * w, 1)
    r_in = 0.5 * np.cos(np.arctan(1 / 2) / 2) ** 2 * 0.95       # well inside every face
    def meets(r):
        disc = b * b - (np.sum(o * o, 1) - r * r)
        return alive & (disc > 0) & (-b - np.sqrt(np.maximum(disc, 0)) > 0)
    lo = meets(r_in).reshape(-1, spp).sum(1)
    hi = meets(0.5 * 1.0001).reshape(-1, spp).sum(1)
    assert (kk >= lo).all() and (kk <= hi).all() and (kk > 0).mean() > 0.2
