"""Pins of the FP64 labelling oracle: closed forms on a single triangle and a cube,
a linear-solve restatement of the ray/plane system, the analytic-sphere bracket on an
icosphere and the t-shift invariant of Eq. 2 (phi(x) - phi(x + t theta) = t)."""

import numpy as np

from ddf_synth import icosphere, torus_knot, uniform_sphere_rays
from oracle.label import label_rays, mt_pairs
from oracle.sphere import sphere_ddf

TRI = (np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), np.array([[0, 1, 2]], np.int32))


def _down(xy, z=1.0):
    xy = np.asarray(xy, np.float64)
    o = np.concatenate([xy, np.full((xy.shape[0], 1), z)], 1).astype(np.float32)
    w = np.tile(np.array([[0, 0, -1]], np.float32), (xy.shape[0], 1))
    return o, w


def test_single_triangle_closed_form():
    V, F = TRI
    pts = [(0.25, 0.25), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5), (0, 0), (1, 0), (0, 1),
           (0.6, 0.5), (-1e-7, 0.5), (0.5, -1e-7), (2, 2)]
    expect = [1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0]
    o, w = _down(pts)
    d, h, t, _ = label_rays(V, F, o, w)
    assert h.tolist() == expect
    assert (d[h == 1] == 1.0).all()
    assert np.isinf(d[h == 0]).all() and (t[h == 0] == -1).all() and (t[h == 1] == 0).all()


def test_single_triangle_behind_and_parallel():
    V, F = TRI
    o = np.array([[0.2, 0.2, -1.0], [0.2, 0.2, 0.0], [0.2, 0.2, 1.0]], np.float32)
    w = np.array([[0, 0, -1], [1, 0, 0], [0, 0, 1]], np.float32)
    d, h, t, _ = label_rays(V, F, o, w)
    assert h.tolist() == [0, 0, 0]          # behind (t < 0), parallel (det = 0), away


def _cube():
    c = np.array([[x, y, z] for x in (-0.5, 0.5) for y in (-0.5, 0.5) for z in (-0.5, 0.5)], np.float32)
    idx = {tuple(v): i for i, v in enumerate(c.tolist())}
    F = []
    for ax in range(3):
        for s in (-0.5, 0.5):
            quad = []
            for a in (-0.5, 0.5):
                for b in (-0.5, 0.5):
                    p = [0.0, 0.0, 0.0]
                    p[ax] = s
                    p[(ax + 1) % 3] = a
                    p[(ax + 2) % 3] = b
                    quad.append(idx[tuple(p)])
            F += [[quad[0], quad[1], quad[3]], [quad[0], quad[3], quad[2]]]
    return c, np.array(F, np.int32)


def test_cube_hand_computed():
    V, F = _cube()
    o = np.array([[0.1, 0.2, 2.0], [-3.0, 0.1, 0.3], [0.0, 0.0, 0.0], [0.7, 0.0, 2.0],
                  [0.3, -0.2, -1.25]], np.float32)
    w = np.array([[0, 0, -1], [1, 0, 0], [1, 0, 0], [0, 0, -1], [0, 0, 1]], np.float32)
    d, h, t, _ = label_rays(V, F, o, w)
    assert h.tolist() == [1, 1, 1, 0, 1]
    assert np.allclose(d[[0, 1, 2, 4]], [1.5, 2.5, 0.5, 0.75], rtol=0, atol=1e-7)
    # the face that was hit lies in the plane the ray reached
    for k in (0, 1, 2, 4):
        tri = V[F[t[k]]].astype(np.float64)
        q = o[k].astype(np.float64) + float(d[k]) * w[k].astype(np.float64)
        nrm = np.cross(tri[1] - tri[0], tri[2] - tri[0])
        assert abs(np.dot(q - tri[0], nrm)) < 1e-6


def test_shared_edge_tie_goes_to_lowest_index():
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], np.float32)
    for F in (np.array([[0, 1, 2], [0, 2, 3]], np.int32), np.array([[0, 2, 3], [0, 1, 2]], np.int32)):
        o, w = _down([(0.5, 0.5), (0.25, 0.25)])
        d, h, t, _ = label_rays(V, F, o, w)
        assert h.tolist() == [1, 1] and t.tolist() == [0, 0]
        assert d.tolist() == [1.0, 1.0]


def test_mt_matches_linear_solve():
    """MT's (u, v, t) equal the solution of o + t w = v0 + u e1 + v e2 by LAPACK."""
    rng = np.random.default_rng(5)
    n = 2000
    v0, v1, v2 = (rng.uniform(-1, 1, (n, 3)) for _ in range(3))
    o = rng.uniform(-2, 2, (n, 3))
    ab = rng.uniform(-0.3, 1.0, (n, 2))
    tgt = v0 + ab[:, :1] * (v1 - v0) + ab[:, 1:] * (v2 - v0)
    w = tgt - o
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    w[::3] *= -1.0                                         # some rays point away (t < 0)
    hit, t = mt_pairs(o, w, v0, v1, v2)
    A = np.stack([-w, v1 - v0, v2 - v0], axis=2)          # columns: -w, e1, e2
    sol = np.linalg.solve(A, (o - v0)[..., None])[..., 0]  # (t, u, v)
    ts, us, vs = sol[:, 0], sol[:, 1], sol[:, 2]
    assert np.allclose(t, ts, rtol=1e-9, atol=1e-9)
    margin = 1e-9
    clear = (np.minimum(np.minimum(us, vs), 1 - us - vs) > margin) | \
            (np.minimum(np.minimum(us, vs), 1 - us - vs) < -margin)
    clear &= np.abs(ts) > margin
    ref = (us >= 0) & (vs >= 0) & (us + vs <= 1) & (ts > 0)
    assert (hit[clear] == ref[clear]).all()
    assert ref.sum() > 50 and (~ref).sum() > 50


def test_icosphere_sphere_bracket():
    R = 0.5
    V, F = icosphere(2, R)
    Vd = V.astype(np.float64)
    tri = Vd[F]
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r_in = float(np.min(np.abs(np.sum(nrm * tri[:, 0], axis=1))))
    assert 0.48 < r_in < R
    o, w = uniform_sphere_rays(4096, seed=3)
    d, h, t, t64 = label_rays(V, F, o, w)
    o64, w64 = o.astype(np.float64), w.astype(np.float64)
    b = np.sum(o64 * w64, 1)
    imp = np.sqrt(np.maximum(0, np.sum(o64 * o64, 1) - b * b))
    front = b < 0
    inner = front & (imp < r_in - 1e-9)
    outer = (imp > R + 1e-9) | ~front
    assert h[inner].all() and not h[outer].any()
    assert inner.sum() > 100
    d_out, _, _ = sphere_ddf(o64[inner], w64[inner], R)
    d_in, _, _ = sphere_ddf(o64[inner], w64[inner], r_in)
    assert (d_out <= t64[inner] + 1e-12).all() and (t64[inner] <= d_in + 1e-12).all()


def test_t_shift_invariant_eq2():
    V, F = torus_knot(3, 2, 0.08, 64, 8)
    o, w = uniform_sphere_rays(3000, seed=9)
    d, h, t, t64 = label_rays(V, F, o, w)
    k = np.nonzero(h)[0][:300]
    assert k.size > 100
    rng = np.random.default_rng(1)
    frac = rng.uniform(0.0, 0.9, k.size)
    Vd = V.astype(np.float64)
    from oracle.label import mt_pairs as mt
    v0, v1, v2 = Vd[F[:, 0]], Vd[F[:, 1]], Vd[F[:, 2]]
    for j, i in enumerate(k):
        s = frac[j] * t64[i]
        o2 = o[i].astype(np.float64) + s * w[i].astype(np.float64)
        hit, tt = mt(o2[None], w[i].astype(np.float64)[None], v0, v1, v2)
        tt = np.where(hit, tt, np.inf)
        jj = int(np.argmin(tt))
        assert jj == t[i]
        assert abs(tt[jj] - (t64[i] - s)) <= 1e-12 * (1 + t64[i])
