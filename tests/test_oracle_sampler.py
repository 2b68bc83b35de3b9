"""Pins of the surface-marching sampler oracle (Sec. 5.2, Eqs. 8-12, odd-even inside test)
against facts that hold independently of it: the series against numpy's sin / cos, Eq. 9's
angle naming, face points on their faces, the odd-even rule on a convex mesh (a point just
outside the surface crosses it zero times, one just inside once; a ray leaving a convex body
never meets it again), and, on a non-convex scene of two spheres, the marching limit (every
Eq. 10 sample's own ray meets its face point first, which fails if the march runs past the first
hit) and the infinite-field samples (their rays meet nothing)."""

import numpy as np
import pytest

from ddf_synth import icosphere
from oracle import sampler as S
from oracle.label import label_rays


def test_sincospi_series_matches_numpy():
    u = np.arange(-2 ** 26, 2 ** 26, 4099, dtype=np.float64) * 2.0 ** -25   # multiples of 2^-25 in [-2, 2)
    s, c = S.sincospi(u)
    # numpy's sin(pi u) carries the rounding of pi u (up to ~7e-16 at |u| = 2)
    assert np.abs(s - np.sin(np.pi * u)).max() < 1.5e-15
    assert np.abs(c - np.cos(np.pi * u)).max() < 1.5e-15
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    for x, sx, cx in zip(u[::400], s[::400], c[::400]):   # against 120-bit sin / cos
        assert abs(float(mpmath.sinpi(mpmath.mpf(x))) - sx) < 2.5e-16
        assert abs(float(mpmath.cospi(mpmath.mpf(x))) - cx) < 2.5e-16
    # exact values at the quadrant points
    s, c = S.sincospi(np.array([0.0, 0.5, 1.0, 1.5]))
    assert np.array_equal(s, [0.0, 1.0, 0.0, -1.0]) and np.array_equal(c, [1.0, 0.0, -1.0, 0.0])


def test_eq9_names_polar_and_azimuth():
    d = S.direction(np.float32([0.0, 0.5, 0.5, 1.0]), np.float32([0.3, 0.0, 0.25, 0.7]))
    assert np.allclose(d[0], [0, 0, 1], atol=1e-7)          # theta_0 = 0: the +z pole
    assert np.allclose(d[1], [1, 0, 0], atol=1e-7)          # theta_0 = pi/2, theta_1 = 0: +x
    assert np.allclose(d[2], [0, 1, 0], atol=1e-7)          # theta_1 = pi/2: +y
    assert np.allclose(d[3], [0, 0, -1], atol=1e-7)
    assert d.dtype == np.float32


def test_face_points_lie_on_their_faces_uniformly():
    V, T = icosphere(1, 0.5)
    P = S.face_points(V, T, 64, seed=5).astype(np.float64)
    F = np.repeat(np.arange(T.shape[0]), 64)
    v0, v1, v2 = (V[T[F, j]].astype(np.float64) for j in range(3))
    # barycentric coordinates by least squares in the face plane
    M = np.stack([v1 - v0, v2 - v0], axis=2)                       # (n, 3, 2)
    ab = np.linalg.lstsq(M[0], (P - v0)[0], rcond=None)[0]
    ab = np.stack([np.linalg.lstsq(M[i], P[i] - v0[i], rcond=None)[0] for i in range(P.shape[0])])
    resid = np.einsum("nij,nj->ni", M, ab) - (P - v0)
    assert np.abs(resid).max() < 1e-6
    assert ab.min() > -1e-5 and (ab.sum(1)).max() < 1 + 1e-5
    assert abs(ab[:, 0].mean() - 1 / 3) < 0.02 and abs(ab[:, 1].mean() - 1 / 3) < 0.02


def test_odd_even_rule_on_a_convex_mesh():
    V, T = icosphere(2, 0.5)
    r = S.sample_surface(V, T, s_fc=2, s_dr=4, s_p=4, eps=1e-4, seed=11)
    Vd = V.astype(np.float64)
    n = np.cross(Vd[T[:, 1]] - Vd[T[:, 0]], Vd[T[:, 2]] - Vd[T[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    face = np.repeat(np.arange(T.shape[0]), 2 * 4)
    cosn = np.sum(r["cand_dir"].astype(np.float64) * n[face], axis=1)
    clear = np.abs(cosn) > 1e-2
    assert clear.mean() > 0.95
    # inward directions start inside: one crossing; outward ones none, and never hit again
    assert np.array_equal(r["cand_parity"][clear], (cosn[clear] < 0).astype(np.uint8))
    out = clear & (cosn > 0)
    assert (r["cand_hit"][out] == 0).all()
    # every kept candidate of a convex body misses: each gives s_p samples of Eq. 10 and Eq. 11
    kinds = r["key"] % 4
    kept = int(out.sum())
    assert (kinds == 0).sum() >= kept * 4 and (kinds == 1).sum() >= kept * 4


def _two_spheres():
    Va, Ta = icosphere(2, 0.3)
    Vb = Va.copy()
    Va = Va + np.float32([-0.45, 0.0, 0.0])
    Vb = Vb + np.float32([0.45, 0.0, 0.0])
    return np.concatenate([Va, Vb]).astype(np.float32), np.concatenate([Ta, Ta + Va.shape[0]]).astype(np.int32)


@pytest.fixture(scope="module")
def two_spheres_samples():
    V, T = _two_spheres()
    return V, T, S.sample_surface(V, T, s_fc=1, s_dr=6, s_p=5, eps=1e-4, seed=3)


def test_marching_stops_at_the_first_hit(two_spheres_samples):
    V, T, r = two_spheres_samples
    k0 = r["key"] % 4 == 0
    assert k0.sum() > 1000
    # rays of one sphere that meet the other were marched, and only up to that hit
    assert ((r["cand_hit"] == 1) & (r["cand_parity"] == 0)).sum() > 20
    d, h, tri, _ = label_rays(V, T, r["o"][k0], r["w"][k0])
    assert (h == 1).all()
    # the first surface along -theta is the candidate's own face, at the marched distance (up to
    # the float32 rounding of q, amplified at grazing angles)
    face = (r["key"][k0] // 4) // 5 // 6
    assert np.mean(tri == face) > 0.995
    assert np.abs(d - r["dist"][k0]).max() < 1e-4


def test_infinite_field_samples_meet_nothing(two_spheres_samples):
    V, T, r = two_spheres_samples
    inf = r["key"] % 4 != 0
    assert inf.sum() > 500 and ((r["key"] % 4) >= 2).sum() > 100
    assert np.isinf(r["dist"][inf]).all() and (r["hit"][inf] == 0).all()
    _, h, _, _ = label_rays(V, T, r["o"][inf], r["w"][inf])
    assert (h == 0).all()
    # Eq. 12 directions are perpendicular to their ray
    c = r["key"] // 4 // 5
    perp = (r["key"] % 4) >= 2
    th = r["cand_dir"][c[perp]].astype(np.float64)
    assert np.abs(np.sum(th * r["w"][perp], axis=1)).max() < 1e-6


def test_keys_are_sorted_and_unique(two_spheres_samples):
    _, _, r = two_spheres_samples
    assert np.all(np.diff(r["key"]) > 0)
