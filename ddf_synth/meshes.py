"""Procedural closed triangle meshes standing in for the paper's ShapeNet / bunny / Suzanne
objects (which are not available): icospheres, tori and (p, q) torus knots, all placed
inside the unit ball that serves as the DDF's bounding domain B (Sec. 3.1).

Vertices are built in float64 and rounded to float32 once; triangles are int32 with
counter-clockwise winding seen from outside (outward normals).
"""

from __future__ import annotations

import numpy as np


def _finish(verts64: np.ndarray, tris: np.ndarray):
    v32 = np.ascontiguousarray(verts64.astype(np.float32))
    t32 = np.ascontiguousarray(tris.astype(np.int32))
    return v32, t32


def icosphere(level: int = 2, radius: float = 0.5):
    """Icosahedron subdivided `level` times, every vertex projected onto the sphere of
    `radius` centred at the origin. Triangle count is 20 * 4**level (level 2 -> 320)."""
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = [
        (-1, phi, 0), (1, phi, 0), (-1, -phi, 0), (1, -phi, 0),
        (0, -1, phi), (0, 1, phi), (0, -1, -phi), (0, 1, -phi),
        (phi, 0, -1), (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1),
    ]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [
        (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
        (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
        (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
        (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
    ]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.stack(verts) * radius
    F = np.array(faces, dtype=np.int64)
    return _finish(V, F)


def _grid_tris(nu: int, nv: int) -> np.ndarray:
    """Two triangles per cell of a periodic nu x nv grid (vertex index i*nv + j)."""
    i = np.arange(nu)[:, None]
    j = np.arange(nv)[None, :]
    a = i * nv + j
    b = ((i + 1) % nu) * nv + j
    c = ((i + 1) % nu) * nv + (j + 1) % nv
    d = i * nv + (j + 1) % nv
    t1 = np.stack([a, b, c], -1).reshape(-1, 3)
    t2 = np.stack([a, c, d], -1).reshape(-1, 3)
    out = np.empty((t1.shape[0] * 2, 3), dtype=np.int64)
    out[0::2] = t1
    out[1::2] = t2
    return out


def torus(major: float = 0.6, minor: float = 0.25, nu: int = 32, nv: int = 16):
    """Torus around the z axis; 2 * nu * nv triangles."""
    u = 2.0 * np.pi * np.arange(nu) / nu
    w = 2.0 * np.pi * np.arange(nv) / nv
    U, W = np.meshgrid(u, w, indexing="ij")
    x = (major + minor * np.cos(W)) * np.cos(U)
    y = (major + minor * np.cos(W)) * np.sin(U)
    z = minor * np.sin(W)
    V = np.stack([x, y, z], -1).reshape(-1, 3)
    return _finish(V, _grid_tris(nu, nv))


def torus_knot(p: int = 3, q: int = 2, tube: float = 0.08, n_seg: int = 256, n_ring: int = 16,
               max_radius: float = 0.95):
    """Tube of radius `tube` around the (p, q) torus-knot centre line
    c(s) = ((2 + cos qs) cos ps, (2 + cos qs) sin ps, -sin qs), scaled so that the
    whole mesh fits in the ball of radius `max_radius`. The tube frame at each
    centre-line point is N = normalised component of c orthogonal to the tangent,
    B = T x N (c is never parallel to T on this curve, so the frame is smooth).
    2 * n_seg * n_ring triangles (256 x 16 -> 8,192; 1,024 x 64 -> 131,072)."""
    s = 2.0 * np.pi * np.arange(n_seg) / n_seg
    r = 2.0 + np.cos(q * s)
    c = np.stack([r * np.cos(p * s), r * np.sin(p * s), -np.sin(q * s)], -1)
    dr = -q * np.sin(q * s)
    dc = np.stack([dr * np.cos(p * s) - r * p * np.sin(p * s),
                   dr * np.sin(p * s) + r * p * np.cos(p * s),
                   -q * np.cos(q * s)], -1)
    T = dc / np.linalg.norm(dc, axis=1, keepdims=True)
    N = c - np.sum(c * T, axis=1, keepdims=True) * T
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    B = np.cross(T, N)
    # scale: centre line reaches |c| <= 3; choose k so that k*3 + tube <= max_radius
    k = (max_radius - tube) / float(np.max(np.linalg.norm(c, axis=1)))
    ang = 2.0 * np.pi * np.arange(n_ring) / n_ring
    ca, sa = np.cos(ang), np.sin(ang)
    V = (k * c[:, None, :]
         + tube * (ca[None, :, None] * N[:, None, :] + sa[None, :, None] * B[:, None, :]))
    V = V.reshape(-1, 3)
    F = _grid_tris(n_seg, n_ring)
    # make the winding outward: the first triangle's normal must point away from the tube axis
    v0, v1, v2 = V[F[0, 0]], V[F[0, 1]], V[F[0, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    if np.dot(nrm, v0 - k * c[0]) < 0:
        F = F[:, [0, 2, 1]]
    return _finish(V, F)


def mesh_euler_characteristic(verts: np.ndarray, tris: np.ndarray) -> int:
    """V - E + F of the triangle mesh (2 for a sphere, 0 for a torus or knot tube)."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e.sort(axis=1)
    n_edges = np.unique(e, axis=0).shape[0]
    n_verts = np.unique(tris).shape[0]
    return int(n_verts - n_edges + tris.shape[0])
