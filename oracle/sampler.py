"""The training-set samplers: surface marching of Sec. 5.2 (Eqs. 8-12) with the odd-even inside
test, and the point-of-view baseline of Sec. 6 (at the end of this module), in float64 where
they decide and in a stated float32 order where they produce coordinates. Test infrastructure
only (see the package docstring).

For every face, s_fc points (Eq. 8); for every point, s_dr directions (Eq. 9); every (point,
direction) ray is marched and the field values along it are collected (Eqs. 10-12):

* the ray is cast from p + eps theta along theta: its nearest hit t1 and the parity of its
  crossings (every hit with t > 0, the labelling test of ``oracle.label``) come from float64
  Moeller-Trumbore on the float32 inputs. An odd parity means the ray starts inside the mesh
  (the odd-even rule: the ray ends outside the bounding box, where every point is outside) and
  the ray is dropped (the field is not defined inside);
* march points q_k = p + t_k theta, t_k = t_end k / (s_p + 1), k = 1 .. s_p, with t_end the hit
  distance eps + t1, or, for a ray that hits nothing, the distance to the unit sphere (the scene
  bound) along theta;
* Eq. 10: (q_k, -theta; t_k), a hit at distance t_k (the face point p);
* for a ray that hits nothing, Eq. 11: (q_k, theta; inf) and Eq. 12: (q_k, theta_perp; inf) for
  the two directions at polar angle theta_0 +- pi/2 (same azimuth) whose own ray from q_k hits no
  face.

Readings (the paper is silent or garbled):

* Eq. 8 as printed leaves the face when a + b > 1; such a pair is reflected to (1 - a, 1 - b),
  which keeps the point uniform on the face.
* s_fc counts points per face, s_dr directions per point, s_p march points per ray; the march
  points split (0, t_end) evenly, end points excluded.
* Eq. 9: theta_0 = a pi is the polar angle, theta_1 = 2 b pi the azimuth, theta =
  (sin th0 cos th1, sin th0 sin th1, cos th0) (the paper's Eq. 9 names are used; it is not
  uniform on the sphere, as printed).
* "theta +- pi/2" (Eq. 12) is the polar angle +- pi/2 at the same azimuth.
* The random numbers: Philox4x32-10 with key = seed; the face point of (face f, point i) uses
  counter (f s_fc + i, 0, 2, 0) and the direction of candidate c = (f s_fc + i) s_dr + j uses
  counter (c, 0, 3, 0) (64-bit indices as low / high words); u = (word >> 8) 2^-24.
* Coordinates are float32, computed in this order without fused multiply-adds:
  p = ((1 - a - b) p0 + a p1) + b p2 per coordinate; the ray origin p + eps theta; q_k =
  p + t_k theta; t_k = t_end * float32(k / (s_p + 1)). sin and cos of an angle u pi (u a
  multiple of 2^-24 or 2^-25) come from ``sincospi``: an exact reduction of u to r in
  [-1/4, 1/4] and Taylor series of sin(pi r) and cos(pi r) in float64 in a fixed order, rounded
  to float32 at the end (the GPU evaluates the same series). t_end for a miss is
  -b + sqrt(b^2 - c), b = p.theta, c = |p|^2 - 1 (dot products summed x, y, then z), in float64
  rounded to float32.
* Every sample carries a key ((c s_p + k - 1) 4 + kind), kind 0 for Eq. 10, 1 for Eq. 11, 2 and 3
  for Eq. 12 (+ then -); samples come out in key order.
"""

from __future__ import annotations

import numpy as np

from .label import label_rays, mt_pairs
from .philox import MASK, philox4x32_10

PI64 = 3.141592653589793   # float64 pi


def _uniforms(seed: int, idx: np.ndarray, stream: int) -> np.ndarray:
    """The first two Philox words of counter (idx lo, idx hi, stream, 0), as u = (w >> 8) 2^-24
    in float32 (exact)."""
    idx = np.asarray(idx, dtype=np.uint64)
    ctr = np.stack([idx & MASK, idx >> np.uint64(32), np.full_like(idx, stream), np.zeros_like(idx)], axis=1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    wds = philox4x32_10(ctr, key)
    return ((wds[:, :2] >> np.uint32(8)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def sincospi(u):
    """(sin(pi u), cos(pi u)) for float64 u that are multiples of 2^-25: u is reduced exactly to
    r = u - n / 2 in [-1/4, 1/4] (n = round(2 u)), x = pi r in float64, Taylor series of sin x to
    x^21 and cos x to x^22 evaluated by Horner's rule from the highest term, then rotated by the
    quadrant n mod 4. The result is float64 (callers round to float32)."""
    u = np.asarray(u, np.float64)
    n = np.floor(2.0 * u + 0.5)
    r = u - 0.5 * n
    x = r * PI64
    x2 = x * x
    s = np.zeros_like(x)
    for k in range(10, -1, -1):          # sin x = sum_k (-1)^k x^(2k+1) / (2k+1)!
        s = s * x2 + ((-1.0) ** k) / _fact(2 * k + 1)
    s = s * x
    c = np.zeros_like(x)
    for k in range(11, -1, -1):          # cos x = sum_k (-1)^k x^(2k) / (2k)!
        c = c * x2 + ((-1.0) ** k) / _fact(2 * k)
    q = (n.astype(np.int64) % 4 + 4) % 4
    sin = np.where(q == 0, s, np.where(q == 1, c, np.where(q == 2, -s, -c)))
    cos = np.where(q == 0, c, np.where(q == 1, -s, np.where(q == 2, -c, s)))
    return sin, cos


def _fact(k):
    f = 1.0
    for i in range(2, k + 1):
        f *= i
    return f


def direction(u0, u1):
    """Eq. 9: theta_0 = u0 pi (polar), theta_1 = 2 u1 pi (azimuth); float32 unit vector."""
    s0, c0 = sincospi(np.asarray(u0, np.float64))
    s1, c1 = sincospi(2.0 * np.asarray(u1, np.float64))
    return np.stack([(s0 * c1).astype(np.float32), (s0 * s1).astype(np.float32), c0.astype(np.float32)], axis=-1)


def face_points(verts, tris, s_fc: int, seed: int):
    """Eq. 8 with the reflection reading: (T s_fc, 3) float32 points, point i of face f at row
    f s_fc + i."""
    V = np.asarray(verts, np.float32)
    F = np.asarray(tris, np.int64)
    T = F.shape[0]
    idx = np.arange(T * s_fc, dtype=np.uint64)
    ab = _uniforms(seed, idx, 2)
    a, b = ab[:, 0].copy(), ab[:, 1].copy()
    flip = (a.astype(np.float64) + b.astype(np.float64)) > 1.0
    a[flip] = np.float32(1.0) - a[flip]
    b[flip] = np.float32(1.0) - b[flip]
    w0 = (np.float32(1.0) - a) - b                       # exact: multiples of 2^-24 in [0, 1]
    f = (idx // np.uint64(s_fc)).astype(np.int64)
    p0, p1, p2 = V[F[f, 0]], V[F[f, 1]], V[F[f, 2]]
    return (w0[:, None] * p0 + a[:, None] * p1) + b[:, None] * p2   # float32 ops, no FMA


def crossing_parity(verts, tris, o, w, chunk_elems: int = 1 << 22):
    """Parity (0 / 1) of the number of faces the rays (o, w) hit at t > 0 (float64
    Moeller-Trumbore of ``oracle.label``), the odd-even inside test."""
    V = np.asarray(verts, np.float32).astype(np.float64)
    F = np.asarray(tris, np.int64)
    v0, v1, v2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    o = np.asarray(o, np.float32).astype(np.float64)
    w = np.asarray(w, np.float32).astype(np.float64)
    n, T = o.shape[0], F.shape[0]
    out = np.zeros(n, np.int64)
    rows = max(1, chunk_elems // max(T, 1))
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        hit, _ = mt_pairs(o[r0:r1, None, :], w[r0:r1, None, :], v0[None], v1[None], v2[None])
        out[r0:r1] = hit.sum(axis=1)
    return (out & 1).astype(np.uint8)


def sample_surface(verts, tris, s_fc: int, s_dr: int, s_p: int, eps: float, seed: int):
    """The dataset of Eqs. 10-12: dict of o (n, 3), w (n, 3), dist (n,) float32 (inf for the
    infinite-field samples), hit (n,) uint8 and key (n,) int64, in key order; also the
    candidates' parity and nearest-hit flag for inspection."""
    V = np.asarray(verts, np.float32)
    F = np.asarray(tris, np.int64)
    T = F.shape[0]
    P = face_points(V, F, s_fc, seed)                                  # (T s_fc, 3)
    C = T * s_fc * s_dr
    cidx = np.arange(C, dtype=np.uint64)
    u = _uniforms(seed, cidx, 3)
    th = direction(u[:, 0], u[:, 1])                                   # (C, 3)
    p = np.repeat(P, s_dr, axis=0)                                     # point of candidate c
    e32 = np.float32(eps)
    ro = p + e32 * th                                                  # float32
    dist1, hit1, _, _ = label_rays(V, F, ro, th)
    par = crossing_parity(V, F, ro, th)
    # t_end: the hit distance from p, or the exit through the unit sphere for a miss
    p64, th64 = p.astype(np.float64), th.astype(np.float64)
    bq = (p64[:, 0] * th64[:, 0] + p64[:, 1] * th64[:, 1]) + p64[:, 2] * th64[:, 2]
    cq = ((p64[:, 0] * p64[:, 0] + p64[:, 1] * p64[:, 1]) + p64[:, 2] * p64[:, 2]) - 1.0
    with np.errstate(invalid="ignore"):
        t_exit = (-bq + np.sqrt(bq * bq - cq)).astype(np.float32)
    t_end = np.where(hit1 == 1, e32 + dist1, t_exit).astype(np.float32)
    valid = (par == 0) & np.isfinite(t_end) & (t_end > 0)
    frac = (np.arange(1, s_p + 1, dtype=np.float32) / np.float32(s_p + 1)).astype(np.float32)
    tk = t_end[:, None] * frac[None, :]                                # (C, s_p) float32
    q = p[:, None, :] + tk[:, :, None] * th[:, None, :]                # (C, s_p, 3) float32
    keys0 = (np.arange(C, dtype=np.int64)[:, None] * s_p + np.arange(s_p)[None, :]) * 4
    miss = valid & (hit1 == 0)
    # Eq. 12 candidates: polar angle +- pi/2
    perp = []
    for sgn in (1.0, -1.0):
        perp.append(direction(u[:, 0].astype(np.float64) + sgn * 0.5, u[:, 1]))
    out = {"o": [], "w": [], "dist": [], "hit": [], "key": []}

    def emit(mask, oo, ww, dd, hh, kk):
        out["o"].append(oo[mask])
        out["w"].append(ww[mask])
        out["dist"].append(dd[mask])
        out["hit"].append(hh[mask])
        out["key"].append(kk[mask])

    flat = lambda a: a.reshape(-1, *a.shape[2:])   # noqa: E731
    vmask = np.repeat(valid, s_p)
    mmask = np.repeat(miss, s_p)
    qf = flat(q)
    thf = np.repeat(th, s_p, axis=0)
    emit(vmask, qf, -thf, tk.reshape(-1), np.ones(C * s_p, np.uint8), keys0.reshape(-1))
    emit(mmask, qf, thf, np.full(C * s_p, np.inf, np.float32), np.zeros(C * s_p, np.uint8), keys0.reshape(-1) + 1)
    for m, pd in enumerate(perp):
        pdf = np.repeat(pd, s_p, axis=0)
        sel = np.nonzero(mmask)[0]
        free = np.zeros(C * s_p, bool)
        if sel.size:
            _, ph, _, _ = label_rays(V, F, qf[sel], pdf[sel])
            free[sel] = ph == 0
        emit(free, qf, pdf, np.full(C * s_p, np.inf, np.float32), np.zeros(C * s_p, np.uint8),
             keys0.reshape(-1) + 2 + m)
    res = {k: np.concatenate(v) for k, v in out.items()}
    order = np.argsort(res["key"], kind="stable")
    res = {k: v[order] for k, v in res.items()}
    res["cand_parity"] = par
    res["cand_hit"] = hit1
    res["cand_dir"] = th
    res["cand_point"] = p
    return res


# --------------------------------------------------------------------------- POV sampling
# The point-of-view baseline of Sec. 6 (Fig. 6's "pov" curve): cameras spaced uniformly in
# azimuth and polar angle around the mesh centre, aimed at it; every pixel's ray is labelled.
#
# Readings (the paper gives only the camera counts, 10 x 5):
# * camera (i, j), i < n_az, j < n_pol, has azimuth phi_i = 2 pi i / n_az and polar angle
#   theta_j = pi (j + 1) / (n_pol + 1) (uniform, the poles excluded, where the azimuth is
#   degenerate); it sits at distance `dist` from the origin (the mesh lies in the unit ball) and
#   looks at the origin with +z up: eye = dist (s_t c_p, s_t s_p, c_t), forward -eye / dist, right
#   (-s_p, c_p, 0), up (-c_t c_p, -c_t s_p, s_t) (right x up = -forward: a right-handed camera);
# * the film is res x res pixels with tan(fov / 2) = tan_half_fov; pixel (x, y), y counted from
#   the top row, has its ray through the pixel centre: px = ((2x + 1) / res - 1) tan_half_fov,
#   py = (1 - (2y + 1) / res) tan_half_fov;
# * a ray starts where it enters the unit ball (the field's domain, Sec. 3.1), or at the eye if
#   it misses the ball (it then misses the mesh too); its label is the nearest-hit distance from
#   there (the labelling of ``oracle.label``);
# * rays are stored camera by camera (c = j n_az + i), each camera's rows top to bottom.
#
# Arithmetic: sin / cos from ``sincospi`` (its reduction r = u - n / 2 is exact for every u by
# Sterbenz's lemma); eye and frame in float64, rounded to float32 once; px, py in float64,
# rounded once; the unnormalised direction (f + px r) + py u in float32 without fused
# multiply-adds; its length and the division in float64 (sums x, y, z in order); the entry
# distance t0 = max(0, -b - sqrt(b^2 - c)), b = eye.w, c = |eye|^2 - 1, in float64, and the
# origin eye + t0 w in float64, rounded once.


def pov_cameras(n_az: int, n_pol: int, dist: float):
    """(eye, forward, right, up) float32 arrays of shape (n_az n_pol, 3), camera c = j n_az + i."""
    i = np.tile(np.arange(n_az, dtype=np.float64), n_pol)
    j = np.repeat(np.arange(n_pol, dtype=np.float64), n_az)
    sp, cp = sincospi(2.0 * i / float(n_az))
    st, ct = sincospi((j + 1.0) / float(n_pol + 1))
    d = float(np.float32(dist))
    dirv = np.stack([st * cp, st * sp, ct], axis=1)                    # unit vector to the eye
    eye = (d * dirv).astype(np.float32)
    fwd = (-dirv).astype(np.float32)
    right = np.stack([-sp, cp, np.zeros_like(sp)], axis=1).astype(np.float32)
    up = np.stack([-(ct * cp), -(ct * sp), st], axis=1).astype(np.float32)
    return eye, fwd, right, up


def pov_rays(n_az: int, n_pol: int, res: int, dist: float, tan_half_fov: float):
    """Every pixel ray of every camera: float32 origins and unit directions (N, 3), N =
    n_az n_pol res^2, in the stored order."""
    eye, fwd, right, up = pov_cameras(n_az, n_pol, dist)
    th = float(np.float32(tan_half_fov))
    pix = np.arange(res, dtype=np.float64)
    px = (((2.0 * pix + 1.0) / res - 1.0) * th).astype(np.float32)    # by column x
    py = ((1.0 - (2.0 * pix + 1.0) / res) * th).astype(np.float32)    # by row y
    ncam = eye.shape[0]
    PX = np.broadcast_to(px[None, None, :, None], (ncam, res, res, 1))
    PY = np.broadcast_to(py[None, :, None, None], (ncam, res, res, 1))
    F_ = fwd[:, None, None, :]
    R_ = right[:, None, None, :]
    U_ = up[:, None, None, :]
    d = ((F_ + PX * R_) + PY * U_).reshape(-1, 3)                     # float32, no FMA
    d64 = d.astype(np.float64)
    n2 = (d64[:, 0] * d64[:, 0] + d64[:, 1] * d64[:, 1]) + d64[:, 2] * d64[:, 2]
    w = (d64 / np.sqrt(n2)[:, None]).astype(np.float32)
    e = np.repeat(eye, res * res, axis=0).astype(np.float64)
    w64 = w.astype(np.float64)
    b = (e[:, 0] * w64[:, 0] + e[:, 1] * w64[:, 1]) + e[:, 2] * w64[:, 2]
    c = ((e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]) - 1.0
    disc = b * b - c
    with np.errstate(invalid="ignore"):
        sq = np.sqrt(disc)
    enter = (disc > 0.0) & (-b + sq > 0.0)
    t0 = np.where(enter, np.maximum(0.0, -b - sq), 0.0)
    o = (e + t0[:, None] * w64).astype(np.float32)
    return o, w


def sample_pov(verts, tris, n_az: int = 10, n_pol: int = 5, res: int = 64, dist: float = 2.5,
               tan_half_fov: float = 0.2679491924311227):
    """POV samples: dict o, w (N, 3) float32, dist (N,) float32 (inf on a miss), hit (N,) uint8."""
    o, w = pov_rays(n_az, n_pol, res, dist, tan_half_fov)
    d, h, _, _ = label_rays(verts, tris, o, w)
    return {"o": o, "w": w, "dist": d, "hit": h}


# --------------------------------------------------------------------------- random sampling
# The "random" baseline of Sec. 6 (Fig. 6): points and directions picked at random, each ray shot
# into the mesh and its t stored.
#
# Readings: the points are uniform in the bounding box of the field's domain, the cube [-1, 1]^3
# around the unit ball; the directions are uniform on the sphere. Ray i draws Philox counter
# (i, 0, 4, 0) for the point (words 0, 1, 2 -> x, y, z = 2u - 1, exact in float32) and counter
# (i, 0, 5, 0) for the direction (words 0, 1: z = 1 - 2 u0, exact; azimuth 2 pi u1; the planar
# radius sqrt(1 - z^2) in float64, where 1 - z^2 is exact, sines and cosines from ``sincospi``;
# each coordinate rounded to float32 once). The label is the nearest hit of ``oracle.label``.


def _words(seed: int, idx: np.ndarray, stream: int) -> np.ndarray:
    """The four Philox words of counter (idx lo, idx hi, stream, 0) as u = (w >> 8) 2^-24, float64."""
    idx = np.asarray(idx, dtype=np.uint64)
    ctr = np.stack([idx & MASK, idx >> np.uint64(32), np.full_like(idx, stream), np.zeros_like(idx)], axis=1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    return (philox4x32_10(ctr, key) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24


def random_rays(n: int, seed: int):
    """n float32 rays: origins uniform in [-1, 1]^3, unit directions uniform on the sphere."""
    idx = np.arange(n, dtype=np.uint64)
    up = _words(seed, idx, 4)
    o = (2.0 * up[:, :3] - 1.0).astype(np.float32)
    ud = _words(seed, idx, 5)
    z = 1.0 - 2.0 * ud[:, 0]
    r = np.sqrt(1.0 - z * z)
    s, c = sincospi(2.0 * ud[:, 1])
    w = np.stack([(r * c).astype(np.float32), (r * s).astype(np.float32), z.astype(np.float32)], axis=1)
    return o, w


def sample_random(verts, tris, n: int, seed: int):
    """Random samples: dict o, w (n, 3) float32, dist (n,) float32 (inf on a miss), hit (n,) uint8."""
    o, w = random_rays(n, seed)
    d, h, _, _ = label_rays(verts, tris, o, w)
    return {"o": o, "w": w, "dist": d, "hit": h}
