"""Pins of the POV and random sampling oracles (Sec. 6, the "pov" and "random" baselines of
Fig. 6) against facts that hold independently of them: the camera placement against numpy's
trigonometry, an orthonormal right-handed frame, every ray through its pixel centre and starting
on the unit sphere, the centre pixel aimed at the origin, the random rays' moments and
uniformity, and the labels of an axis-aligned cube against the slab method (a closed form that
shares nothing with Moeller-Trumbore)."""

import numpy as np

from oracle import sampler as S

TH = 0.2679491924311227     # tan(15 deg)


def test_cameras_sit_at_the_stated_angles():
    n_az, n_pol, d = 10, 5, 2.5
    eye, fwd, right, up = S.pov_cameras(n_az, n_pol, d)
    assert eye.shape == (50, 3) and eye.dtype == np.float32
    i = np.tile(np.arange(n_az), n_pol)
    j = np.repeat(np.arange(n_pol), n_az)
    phi = 2 * np.pi * i / n_az
    theta = np.pi * (j + 1) / (n_pol + 1)
    ref = d * np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], 1)
    assert np.abs(eye - ref).max() < 4e-7 * d
    assert np.abs(fwd + ref / d).max() < 2e-7
    f, r, u = (x.astype(np.float64) for x in (fwd, right, up))
    for a, b in ((f, r), (f, u), (r, u)):
        assert np.abs(np.sum(a * b, 1)).max() < 1e-6
    for a in (f, r, u):
        assert np.abs(np.linalg.norm(a, axis=1) - 1).max() < 1e-6
    assert np.abs(np.cross(r, u) + f).max() < 1e-6          # right x up = -forward
    assert (u[:, 2] > 0).all()                               # +z up


def test_every_ray_passes_through_its_pixel_centre():
    n_az, n_pol, res, d = 4, 3, 6, 2.5
    o, w = S.pov_rays(n_az, n_pol, res, d, TH)
    assert o.shape == (n_az * n_pol * res * res, 3)
    eye, fwd, right, up = (x.astype(np.float64) for x in S.pov_cameras(n_az, n_pol, d))
    cam = np.repeat(np.arange(n_az * n_pol), res * res)
    y = np.tile(np.repeat(np.arange(res), res), n_az * n_pol)
    x = np.tile(np.arange(res), n_az * n_pol * res)
    px = ((x + 0.5) / res * 2 - 1) * TH
    py = (1 - (y + 0.5) / res * 2) * TH
    aim = fwd[cam] + px[:, None] * right[cam] + py[:, None] * up[cam]
    aim /= np.linalg.norm(aim, axis=1, keepdims=True)
    w64, o64 = w.astype(np.float64), o.astype(np.float64)
    assert np.abs(np.linalg.norm(w64, axis=1) - 1).max() < 1e-6
    assert np.abs(w64 - aim).max() < 1e-6
    # the origin is where the ray from the eye enters the unit ball
    assert np.abs(np.linalg.norm(o64, axis=1) - 1).max() < 1e-6
    back = o64 - eye[cam]
    assert np.abs(np.cross(back, w64)).max() < 1e-5 and (np.sum(back * w64, 1) > 0).all()
    # the top row looks higher than the bottom row (camera at theta = pi / 2 sees +z up)
    top = (cam == 1 * n_az) & (y == 0)
    bottom = (cam == 1 * n_az) & (y == res - 1)
    assert (w64[top, 2] > 0).all() and (w64[bottom, 2] < 0).all()


def test_centre_pixel_is_aimed_at_the_origin():
    o, w = S.pov_rays(3, 2, 9, 2.5, TH)
    c = (np.arange(6) * 81) + 4 * 9 + 4
    o64, w64 = o[c].astype(np.float64), w[c].astype(np.float64)
    assert np.abs(np.cross(o64, w64)).max() < 1e-6
    eye, fwd, _, _ = S.pov_cameras(3, 2, 2.5)
    assert np.array_equal(w[c], fwd) or np.abs(w64 - fwd).max() < 1e-7


def _box(a):
    a = np.float32(a)
    V = np.array([[x, y, z] for x in (-a, a) for y in (-a, a) for z in (-a, a)], np.float32)
    # faces of the box as two triangles each, outward winding
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    F = []
    for q in quads:
        F += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
    return V, np.array(F, np.int32)


def test_cube_labels_match_the_slab_method():
    a = 0.4
    V, F = _box(a)
    r = S.sample_pov(V, F, n_az=10, n_pol=5, res=16)
    o, w = r["o"].astype(np.float64), r["w"].astype(np.float64)
    A = float(np.float32(a))
    with np.errstate(divide="ignore", invalid="ignore"):
        t1, t2 = (-A - o) / w, (A - o) / w
    tn = np.max(np.minimum(t1, t2), axis=1)
    tf = np.min(np.maximum(t1, t2), axis=1)
    hit = (tn <= tf) & (tf > 0)
    # leave out rays within rounding of an edge (the hit point near two faces' planes)
    p = o + tn[:, None] * w
    near_edge = np.sum(np.abs(np.abs(p) - A) < 1e-5, axis=1) >= 2
    grazing = np.abs(tn - tf) < 1e-5
    keep = ~(near_edge | grazing)
    assert keep.mean() > 0.97 and hit.mean() > 0.2 and (~hit).mean() > 0.2
    assert np.array_equal(r["hit"][keep].astype(bool), hit[keep])
    h = keep & hit
    assert np.abs(r["dist"][h] - tn[h]).max() < 1e-6 * (1 + tn[h].max())
    assert np.isinf(r["dist"][keep & ~hit]).all()


def test_random_rays_are_uniform_in_the_box_and_on_the_sphere():
    """The random baseline of Sec. 6: origins fill [-1, 1]^3 uniformly (each coordinate's mean 0,
    variance 1/3, independent), directions are unit and uniform on the sphere (every coordinate's
    mean 0 and second moment 1/3; z and the azimuth each uniform)."""
    n = 200000
    o, w = S.random_rays(n, seed=3)
    assert o.dtype == np.float32 and w.dtype == np.float32
    assert (np.abs(o) <= 1).all()
    assert np.abs(o.mean(0)).max() < 0.01 and np.abs(o.var(0) - 1 / 3).max() < 0.01
    assert np.abs(np.corrcoef(o.T.astype(np.float64))[np.triu_indices(3, 1)]).max() < 0.01
    w64 = w.astype(np.float64)
    assert np.abs(np.linalg.norm(w64, axis=1) - 1).max() < 1e-6
    assert np.abs(w64.mean(0)).max() < 0.01 and np.abs((w64 ** 2).mean(0) - 1 / 3).max() < 0.01
    hz, _ = np.histogram(w64[:, 2], bins=20, range=(-1, 1))
    ha, _ = np.histogram(np.arctan2(w64[:, 1], w64[:, 0]), bins=20, range=(-np.pi, np.pi))
    for h in (hz, ha):
        assert np.abs(h / (n / 20) - 1).max() < 0.05
    # the same seed gives the same rays, another seed others
    o2, w2 = S.random_rays(1000, seed=3)
    assert np.array_equal(o2, o[:1000]) and np.array_equal(w2, w[:1000])
    assert not np.array_equal(S.random_rays(1000, seed=4)[0], o2)


def test_random_samples_on_a_box_match_the_slab_method():
    V, F = _box(0.5)
    r = S.sample_random(V, F, 20000, seed=7)
    o, w = r["o"].astype(np.float64), r["w"].astype(np.float64)
    A = float(np.float32(0.5))
    with np.errstate(divide="ignore", invalid="ignore"):
        t1, t2 = (-A - o) / w, (A - o) / w
    tn = np.max(np.minimum(t1, t2), axis=1)
    tf = np.min(np.maximum(t1, t2), axis=1)
    inside = np.all(np.abs(o) < A, axis=1)
    t = np.where(inside, tf, tn)                     # from inside the box the exit face is hit
    hit = (tn <= tf) & (tf > 0)
    p = o + t[:, None] * w
    edge = np.sum(np.abs(np.abs(p) - A) < 1e-5, axis=1) >= 2
    keep = ~edge & (np.abs(tn - tf) > 1e-5)
    assert keep.mean() > 0.97 and 0.2 < hit.mean() < 0.9
    assert np.array_equal(r["hit"][keep].astype(bool), hit[keep])
    h = keep & hit
    assert np.abs(r["dist"][h] - t[h]).max() < 1e-6 * (1 + t[h].max())
