"""Seeded ray batches for labelling, training and query benchmarks.

A ray is an origin o (float32 x3) and a unit direction w (float32 x3), stored as two
row-major (n, 3) arrays. Origins lie on (or in) the unit ball, the DDF's bounding
domain B (Sec. 3.1). Generation runs in float64 and is rounded to float32 once; the
direction is re-normalised in float64 before rounding, so |w| = 1 to float32 precision.
"""

from __future__ import annotations

import numpy as np


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _uniform_dirs(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform on S^2: z = 1 - 2u, azimuth 2 pi v."""
    u = rng.random(n)
    v = rng.random(n)
    z = 1.0 - 2.0 * u
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    a = 2.0 * np.pi * v
    return np.stack([r * np.cos(a), r * np.sin(a), z], -1)


def _as_f32(o: np.ndarray, w: np.ndarray):
    return (np.ascontiguousarray(o.astype(np.float32)),
            np.ascontiguousarray(_unit(w).astype(np.float32)))


def uniform_sphere_rays(n: int, seed: int, radius: float = 1.0):
    """Origin uniform on the sphere of `radius`, direction uniform on S^2 (independent)."""
    rng = np.random.default_rng(seed)
    o = radius * _uniform_dirs(rng, n)
    w = _uniform_dirs(rng, n)
    return _as_f32(o, w)


def inward_sphere_rays(n: int, seed: int, radius: float = 1.0):
    """Origin uniform on the sphere of `radius`, direction uniform over the inward hemisphere."""
    rng = np.random.default_rng(seed)
    o = radius * _uniform_dirs(rng, n)
    w = _uniform_dirs(rng, n)
    flip = np.sum(w * o, axis=1) > 0
    w[flip] = -w[flip]
    return _as_f32(o, w)


def sample_surface_points(verts: np.ndarray, tris: np.ndarray, n: int, rng: np.random.Generator):
    """Uniform points on the mesh surface: a triangle with probability proportional to its
    area, then barycentric (a, b) ~ U[0,1]^2 reflected to (1-a, 1-b) when a + b > 1 so that
    the point stays on the face (the face sampler of Eq. 8 with that fix)."""
    V = verts.astype(np.float64)
    p0, p1, p2 = V[tris[:, 0]], V[tris[:, 1]], V[tris[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1)
    cdf = np.cumsum(area)
    cdf /= cdf[-1]
    idx = np.searchsorted(cdf, rng.random(n), side="right")
    idx = np.minimum(idx, len(tris) - 1)
    a = rng.random(n)
    b = rng.random(n)
    m = a + b > 1.0
    a[m], b[m] = 1.0 - a[m], 1.0 - b[m]
    pts = (1.0 - a - b)[:, None] * p0[idx] + a[:, None] * p1[idx] + b[:, None] * p2[idx]
    return pts, idx


def _frame(w: np.ndarray):
    """Two unit vectors orthogonal to each unit row of w (any smooth choice)."""
    helper = np.where(np.abs(w[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    t1 = _unit(np.cross(w, helper))
    t2 = np.cross(w, t1)
    return t1, t2


def surface_aimed_rays(verts, tris, n: int, seed: int, sigma: float = 0.05, radius: float = 1.0):
    """Origin uniform on the bounding sphere, aimed at a uniform surface point, then the
    direction is jittered by a Gaussian angle: w' = normalise(w + sigma (g1 t1 + g2 t2))."""
    rng = np.random.default_rng(seed)
    o = radius * _uniform_dirs(rng, n)
    tgt, _ = sample_surface_points(verts, tris, n, rng)
    w = _unit(tgt - o)
    t1, t2 = _frame(w)
    g = rng.standard_normal((n, 2))
    w = _unit(w + sigma * (g[:, :1] * t1 + g[:, 1:] * t2))
    return _as_f32(o, w)


def labelled_ray_set(verts, tris, n: int, seed: int, sigma: float = 0.05):
    """Training-ray mix: half uniform-origin/uniform-direction rays on the bounding sphere,
    half surface-aimed rays with angular jitter `sigma` (interleaved in blocks, seeded)."""
    h = n // 2
    o1, w1 = uniform_sphere_rays(h, seed)
    o2, w2 = surface_aimed_rays(verts, tris, n - h, seed + 1, sigma)
    o = np.concatenate([o1, o2])
    w = np.concatenate([w1, w2])
    perm = np.random.default_rng(seed + 2).permutation(n)
    return np.ascontiguousarray(o[perm]), np.ascontiguousarray(w[perm])


def fibonacci_directions(k: int) -> np.ndarray:
    """k unit directions spread over the sphere (spherical Fibonacci lattice: z uniform in
    (-1, 1), azimuth advancing by the golden angle), float32 (k, 3)."""
    i = np.arange(k, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / k
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * np.pi * (3.0 - np.sqrt(5.0))
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
