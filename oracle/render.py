"""FP64 modified uni-directional path tracer (Sec. 1, Fig. 1): the nearest-surface
search of a classic path tracer is replaced by one DDF query per bounce.
Test infrastructure only (see the package docstring).

The paper gives no pseudo-code; the readings used here:

* Camera: pinhole; forward f = normalise(look_at - eye), right r = normalise(f x up),
  up' = r x f; for pixel (x, y) (row 0 at the top) and jitter (j0, j1),
  dir = normalise(f + px r + py up') with px = (2 (x + j0) / W - 1) tan(vfov/2) W/H and
  py = (1 - 2 (y + j1) / H) tan(vfov/2).
* Path id pid = (y W + x) spp + s. Draws are Philox4x32-10 words of counter
  (pid lo, pid hi, bounce, 0), key = seed; bounce 0 gives the pixel jitter (words 0, 1).
* The DDF is defined for origins in the bounding domain B (Sec. 3.1), the unit ball:
  a primary ray is advanced to its entry point into the unit ball (t0 = max(0, -b -
  sqrt(b^2 - c))); a primary ray that misses the ball (b^2 - c <= 0, or the ball lies
  behind it) returns the environment radiance without a query.
* Bounce b = 1 .. B (B = max queries per path): query (d, logit, n). Miss (logit <= 0):
  radiance = throughput * env, stop. Hit at b = B: radiance = 0, stop. Otherwise the hit
  point q = o + max(d, 0) w (Sec. 3.1, q = x + phi theta), the normal n of Eq. 3, new
  origin q + 1e-4 n, new direction by cosine-weighted hemisphere sampling about n
  (u0, u1 = words 0, 1 of bounce b): local (sqrt(u0) cos 2 pi u1, sqrt(u0) sin 2 pi u1,
  sqrt(1 - u0)) mapped through the orthonormal basis of Duff et al. 2017 ("Building an
  orthonormal basis, revisited"), and throughput *= albedo (Lambertian BRDF albedo/pi,
  cosine pdf cos/pi).
* Pixel value = mean over its spp samples, summed in sample order.
"""

from __future__ import annotations

import math

import numpy as np

from .philox import path_uniforms


def _normalize(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def camera_basis(cam):
    eye = np.array(cam.eye, np.float64)
    f = _normalize(np.array(cam.look_at, np.float64) - eye)
    r = _normalize(np.cross(f, np.array(cam.up, np.float64)))
    u = np.cross(r, f)
    return eye, f, r, u


def primary_rays(cam, pids, spp: int):
    """Primary rays of the given path ids, advanced to the unit ball.
    Returns (o, w, alive) with alive False for rays that miss the ball."""
    pids = np.asarray(pids, np.int64)
    W, H = cam.width, cam.height
    pix = pids // spp
    x = (pix % W).astype(np.float64)
    y = (pix // W).astype(np.float64)
    uni = path_uniforms(cam.seed, pids.astype(np.uint64), 0)
    eye, f, r, u = camera_basis(cam)
    th = math.tan(math.radians(cam.vfov_deg) * 0.5)
    px = (2.0 * (x + uni[:, 0]) / W - 1.0) * th * (W / H)
    py = (1.0 - 2.0 * (y + uni[:, 1]) / H) * th
    d = _normalize(f[None] + px[:, None] * r[None] + py[:, None] * u[None])
    b = d @ eye
    c = float(eye @ eye) - 1.0
    disc = b * b - c
    sq = np.sqrt(np.maximum(disc, 0.0))
    alive = (disc > 0) & (-b + sq > 0)
    t0 = np.maximum(0.0, -b - sq)
    o = eye[None] + t0[:, None] * d
    return o, d, alive


def onb_duff(n):
    """Orthonormal basis (b1, b2) completing unit normals n (Duff et al. 2017)."""
    sign = np.where(n[:, 2] >= 0, 1.0, -1.0)
    a = -1.0 / (sign + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    b1 = np.stack([1.0 + sign * n[:, 0] * n[:, 0] * a, sign * b, -sign * n[:, 0]], -1)
    b2 = np.stack([b, sign + n[:, 1] * n[:, 1] * a, -n[:, 1]], -1)
    return b1, b2


def cosine_direction(n, u0, u1):
    r = np.sqrt(u0)
    phi = 2.0 * np.pi * u1
    lx, ly, lz = r * np.cos(phi), r * np.sin(phi), np.sqrt(1.0 - u0)
    b1, b2 = onb_duff(n)
    return lx[:, None] * b1 + ly[:, None] * b2 + lz[:, None] * n


def shade_step(o, w, d, nm, seed, pids, bounce: int, eps: float = 1e-4):
    """The move of a path that hit at this bounce (Sec. 3.1 and the Lambertian bounce of Fig. 1):
    hit point q = o + max(d, 0) w, new origin q + eps n, new direction cosine-distributed about n
    from the path's Philox draws of this bounce. Returns (origin, direction)."""
    q = o + np.maximum(d, 0.0)[:, None] * w
    uni = path_uniforms(seed, np.asarray(pids, np.int64).astype(np.uint64), bounce)
    return q + eps * nm, cosine_direction(nm, uni[:, 0], uni[:, 1])


def trace_paths(query_fn, cam, spp: int, bounces: int, pids, eps: float = 1e-4):
    """Trace the given paths. query_fn(o, w) -> dict(dist, logit, normal) in float64.

    Returns dict: radiance (per pid), min_abs_logit (smallest |logit| of any hit/miss
    decision taken on the path; +inf if none), first-bounce AOVs (dist, logit, normal,
    queried flag), and rec (n, bounces, 11): every bounce's query ray o, w, its dist, logit
    and normal (NaN where the path did not get that far; the normal NaN on a miss)."""
    pids = np.asarray(pids, np.int64)
    n = pids.size
    rad = np.zeros(n)
    rec = np.full((n, bounces, 11), np.nan)
    min_logit = np.full(n, np.inf)
    aov_d = np.full(n, np.nan)
    aov_l = np.full(n, np.nan)
    aov_n = np.full((n, 3), np.nan)
    o, w, alive = primary_rays(cam, pids, spp)
    rad[~alive] = cam.env
    idx = np.nonzero(alive)[0]
    o, w = o[idx], w[idx]
    thr = np.ones(idx.size)
    for b in range(1, bounces + 1):
        if idx.size == 0:
            break
        res = query_fn(o, w)
        d, lg, nm = res["dist"], res["logit"], res["normal"]
        min_logit[idx] = np.minimum(min_logit[idx], np.abs(lg))
        rec[idx, b - 1, 0:3], rec[idx, b - 1, 3:6] = o, w
        rec[idx, b - 1, 6], rec[idx, b - 1, 7] = d, lg
        if nm is not None:
            h = lg > 0
            rec[idx[h], b - 1, 8:11] = nm[h]
        if b == 1:
            aov_d[idx], aov_l[idx], aov_n[idx] = d, lg, nm
        hit = lg > 0
        miss = ~hit
        rad[idx[miss]] = thr[miss] * cam.env
        if b == bounces:
            rad[idx[hit]] = 0.0
            break
        keep = np.nonzero(hit)[0]
        idx, o, w, d, nm, thr = idx[keep], o[keep], w[keep], d[keep], nm[keep], thr[keep]
        o, w = shade_step(o, w, d, nm, cam.seed, pids[idx], b, eps)
        thr = thr * cam.albedo
    return {"radiance": rad, "min_abs_logit": min_logit, "dist": aov_d, "logit": aov_l,
            "normal": aov_n, "rec": rec}


def render_pixels(query_fn, cam, spp: int, bounces: int, pixels):
    """Per-pixel mean radiance of the listed pixel indices (y W + x), plus per-path info."""
    pixels = np.asarray(pixels, np.int64)
    pids = (pixels[:, None] * spp + np.arange(spp)[None, :]).ravel()
    res = trace_paths(query_fn, cam, spp, bounces, pids)
    rad = res["radiance"].reshape(-1, spp)
    img = np.zeros(pixels.size)
    for s in range(spp):
        img += rad[:, s]
    img /= spp
    res["image"] = img
    res["pids"] = pids
    return res


# --------------------------------------------------------------------------- AOV renders
# The t-value and normal images of Fig. 3 / Fig. 4. Readings: one primary ray per pixel, the
# renderer's camera and bounce-0 jitter with spp = 1 (path id = pixel index); the t-value is the
# distance from the eye to the hit point, |entry - eye| + max(dist, 0) for the field (whose rays
# start where they enter the unit ball), +inf where nothing is hit; the normal is the Eq. 3 normal
# for the field and the unit face normal turned towards the eye for a mesh, 0 on a miss.


def field_aov(query_fn, cam):
    """Depth (H W,), normal (H W, 3) and the |logit| of the hit decision (+inf where the ray
    misses the ball) of the field's AOV render, pixel-major."""
    n = cam.width * cam.height
    pids = np.arange(n, dtype=np.int64)
    o, w, alive = primary_rays(cam, pids, 1)
    eye = np.array(cam.eye, np.float64)
    depth = np.full(n, np.inf)
    normal = np.zeros((n, 3))
    margin = np.full(n, np.inf)
    idx = np.nonzero(alive)[0]
    res = query_fn(o[idx], w[idx])
    hit = res["logit"] > 0
    t0 = np.linalg.norm(o[idx] - eye[None], axis=1)
    h = idx[hit]
    depth[h] = t0[hit] + np.maximum(res["dist"][hit], 0.0)
    normal[h] = res["normal"][hit]
    margin[idx] = np.abs(res["logit"])
    return depth, normal, margin


def mesh_aov(verts, tris, cam):
    """Depth, normal and hit face of the pixel rays cast from the eye against a mesh; the float32
    rays are returned too (o, w)."""
    from .label import label_rays
    n = cam.width * cam.height
    _, w, _ = primary_rays(cam, np.arange(n, dtype=np.int64), 1)
    o = np.broadcast_to(np.array(cam.eye, np.float64), (n, 3)).astype(np.float32)
    w = w.astype(np.float32)
    d, _, tri, _ = label_rays(verts, tris, o, w)
    V = np.asarray(verts, np.float64)
    F = np.asarray(tris, np.int64)
    normal = np.zeros((n, 3))
    h = tri >= 0
    k = F[tri[h]]
    fn = np.cross(V[k[:, 1]] - V[k[:, 0]], V[k[:, 2]] - V[k[:, 0]])
    fn /= np.linalg.norm(fn, axis=1, keepdims=True)
    facing = np.sum(fn * w[h].astype(np.float64), axis=1) > 0
    fn[facing] = -fn[facing]
    normal[h] = fn
    return d.astype(np.float64), normal, tri, o, w


def mesh_query(verts, tris):
    """The path tracer's query with a mesh in place of the field (the "without DDF" renderer of
    Fig. 5): the labeller's nearest hit (float32 rays, as the GPU casts them), logit +1 on a hit and
    -1 on a miss, and the hit face's unit normal turned against the ray."""
    from .label import label_rays
    V = np.asarray(verts, np.float32)
    T = np.asarray(tris, np.int64)
    Vd = V.astype(np.float64)

    def q(o, w):
        d, h, tri, _ = label_rays(V, T, np.asarray(o).astype(np.float32), np.asarray(w).astype(np.float32))
        hit = h == 1
        n = np.zeros((len(d), 3))
        k = T[tri[hit]]
        fn = np.cross(Vd[k[:, 1]] - Vd[k[:, 0]], Vd[k[:, 2]] - Vd[k[:, 0]])
        fn /= np.linalg.norm(fn, axis=1, keepdims=True)
        flip = np.sum(fn * np.asarray(w, np.float64)[hit], axis=1) > 0
        fn[flip] = -fn[flip]
        n[hit] = fn
        return {"dist": np.where(hit, d, 0.0).astype(np.float64), "logit": np.where(hit, 1.0, -1.0), "normal": n}
    return q
