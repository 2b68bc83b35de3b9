"""FP64 ray labelling: nearest ray-triangle hit over all faces of a mesh (the linear
search named in Sec. 1; labels are "shot rays and calculated t", Sec. 6).
Test infrastructure only (see the package docstring).

Per (ray, triangle), Moeller-Trumbore in float64 on the float32 vertices, in this exact
order of operations (each product and sum separately rounded, no fused multiply-add,
dot products summed x, y, then z):

    e1 = v1 - v0,  e2 = v2 - v0
    p  = w x e2 = (wy*e2z - wz*e2y, wz*e2x - wx*e2z, wx*e2y - wy*e2x)
    det = (e1x*px + e1y*py) + e1z*pz,   inv = 1 / det
    s  = o - v0,   u = ((sx*px + sy*py) + sz*pz) * inv
    q  = s x e1,   v = ((wx*qx + wy*qy) + wz*qz) * inv
    t  = ((e2x*qx + e2y*qy) + e2z*qz) * inv
    hit <=> det != 0 and u >= 0 and v >= 0 and (u + v) <= 1 and t > 0

Readings (the paper is silent): barycentric bounds are inclusive, so a ray through a
shared edge meets both faces at the same t; the nearest hit is the minimum t with ties
going to the lowest triangle index; t must be strictly positive; a ray with no hit gets
dist = +inf (the paper's "infinite field value" for invisible oriented points,
Sec. 4.1), hit = 0, tri = -1. The float32 distance is the float64 t rounded to nearest.
"""

from __future__ import annotations

import numpy as np


def mt_pairs(o, w, v0, v1, v2):
    """Moeller-Trumbore for broadcastable float64 arrays (..., 3). Returns (hit, t)."""
    e1x, e1y, e1z = v1[..., 0] - v0[..., 0], v1[..., 1] - v0[..., 1], v1[..., 2] - v0[..., 2]
    e2x, e2y, e2z = v2[..., 0] - v0[..., 0], v2[..., 1] - v0[..., 1], v2[..., 2] - v0[..., 2]
    wx, wy, wz = w[..., 0], w[..., 1], w[..., 2]
    px = wy * e2z - wz * e2y
    py = wz * e2x - wx * e2z
    pz = wx * e2y - wy * e2x
    det = (e1x * px + e1y * py) + e1z * pz
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        inv = 1.0 / det
        sx, sy, sz = o[..., 0] - v0[..., 0], o[..., 1] - v0[..., 1], o[..., 2] - v0[..., 2]
        u = ((sx * px + sy * py) + sz * pz) * inv
        qx = sy * e1z - sz * e1y
        qy = sz * e1x - sx * e1z
        qz = sx * e1y - sy * e1x
        v = ((wx * qx + wy * qy) + wz * qz) * inv
        t = ((e2x * qx + e2y * qy) + e2z * qz) * inv
        hit = (det != 0) & (u >= 0) & (v >= 0) & ((u + v) <= 1.0) & (t > 0)
    return hit, t


def label_rays(verts, tris, o, w, chunk_elems: int = 1 << 22):
    """Brute-force nearest hit of every ray against every triangle.

    verts (V, 3) float32, tris (T, 3) int, o / w (n, 3) float32.
    Returns dist (n,) float32, hit (n,) uint8, tri (n,) int32, t64 (n,) float64."""
    V = np.asarray(verts, np.float32).astype(np.float64)
    F = np.asarray(tris, np.int64)
    v0, v1, v2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    o = np.asarray(o, np.float32).astype(np.float64)
    w = np.asarray(w, np.float32).astype(np.float64)
    n, T = o.shape[0], F.shape[0]
    best_t = np.full(n, np.inf)
    best_i = np.full(n, -1, dtype=np.int64)
    rows = max(1, chunk_elems // max(T, 1))
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        hit, t = mt_pairs(o[r0:r1, None, :], w[r0:r1, None, :], v0[None], v1[None], v2[None])
        tt = np.where(hit, t, np.inf)
        idx = np.argmin(tt, axis=1)            # first minimum -> lowest index on ties
        tmin = tt[np.arange(r1 - r0), idx]
        ok = np.isfinite(tmin)
        best_t[r0:r1] = np.where(ok, tmin, np.inf)
        best_i[r0:r1] = np.where(ok, idx, -1)
    hit = best_i >= 0
    dist = np.where(hit, best_t, np.inf).astype(np.float32)
    return dist, hit.astype(np.uint8), best_i.astype(np.int32), best_t
