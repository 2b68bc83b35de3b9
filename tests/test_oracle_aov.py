"""Pins of the AOV-render oracle (t-value and normal images of Fig. 3 / Fig. 4) against closed
forms computed from the eye, not from the unit-ball entry the renderer starts at: the sphere's
ray-sphere intersection and outward normal, and a box's slab intersection and face normals."""

import numpy as np

from ddf_synth import default_camera
from oracle.render import field_aov, mesh_aov, primary_rays
from oracle.sphere import sphere_ddf
from oracle.mlp import normal_from_gradient


def _sphere_query(r):
    def q(o, w):
        d, hit, g = sphere_ddf(o, w, r)
        return {"dist": np.where(hit, d, 0.0), "logit": np.where(hit, 1.0, -1.0), "normal": normal_from_gradient(g, w)}
    return q


def test_field_aov_of_a_sphere_is_the_ray_sphere_intersection_from_the_eye():
    cam = default_camera(48, 40, seed=3)
    r = 0.45
    depth, normal, _ = field_aov(_sphere_query(r), cam)
    _, w, _ = primary_rays(cam, np.arange(48 * 40), 1)
    e = np.array(cam.eye, np.float64)
    b = w @ e
    c = e @ e - r * r
    disc = b * b - c
    hit = disc > 0
    t = -b - np.sqrt(np.where(hit, disc, 0.0))
    assert 0.1 < hit.mean() < 0.9
    assert np.array_equal(np.isfinite(depth), hit)
    assert np.abs(depth[hit] - t[hit]).max() < 1e-12
    q = e[None] + t[hit][:, None] * w[hit]
    assert np.abs(normal[hit] - q / r).max() < 1e-9
    assert (normal[~hit] == 0).all()


def _box(a):
    a = np.float32(a)
    V = np.array([[x, y, z] for x in (-a, a) for y in (-a, a) for z in (-a, a)], np.float32)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    F = []
    for q in quads:
        F += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
    return V, np.array(F, np.int32)


def test_mesh_aov_of_a_box_is_the_slab_intersection():
    cam = default_camera(40, 40, seed=5)
    V, F = _box(0.35)
    depth, normal, tri, o, w = mesh_aov(V, F, cam)
    o, w = o.astype(np.float64), w.astype(np.float64)
    A = float(np.float32(0.35))
    with np.errstate(divide="ignore"):
        t1, t2 = (-A - o) / w, (A - o) / w
    tn = np.max(np.minimum(t1, t2), 1)
    tf = np.min(np.maximum(t1, t2), 1)
    hit = (tn <= tf) & (tf > 0)
    p = o + tn[:, None] * w
    edge = np.sum(np.abs(np.abs(p) - A) < 1e-6, 1) >= 2
    keep = ~edge
    assert 0.1 < hit.mean() < 0.9
    assert np.array_equal((tri >= 0)[keep], hit[keep])
    h = keep & hit
    assert (np.abs(depth[h] - tn[h]) <= 2.0 ** -23 * tn[h]).all()     # the float32 distance of the labeller
    # the face normal of the entry slab, towards the eye
    ax = np.argmax(np.minimum(t1, t2), 1)
    ref = np.zeros_like(normal)
    ref[np.arange(len(ax)), ax] = -np.sign(w[np.arange(len(ax)), ax])
    assert np.abs(normal[h] - ref[h]).max() < 1e-6
    assert (normal[tri < 0] == 0).all() and np.isinf(depth[tri < 0]).all()
