"""Closed-form DDF of a sphere of radius r centred at the origin (the definitions of
Sec. 3.1 evaluated exactly). Test infrastructure only.

With b = o . w and c = |o|^2 - r^2, the ray meets the sphere iff b^2 - c >= 0; from
outside (c >= 0) the distance is t = -b - sqrt(b^2 - c) and it counts as a hit only if
t > 0; from inside (c < 0) t = -b + sqrt(b^2 - c). The gradient with respect to the
origin is q / sqrt(b^2 - c) from outside and -q / sqrt(b^2 - c) from inside, q = o + t w
the hit point (so Eq. 3 gives the sphere's normal at q, and Eq. 2 holds:
d phi / d o . w = -1).
"""

from __future__ import annotations

import numpy as np


def sphere_ddf(o, w, r: float):
    o = np.asarray(o, np.float64)
    w = np.asarray(w, np.float64)
    b = np.sum(o * w, axis=1)
    c = np.sum(o * o, axis=1) - r * r
    disc = b * b - c
    sq = np.sqrt(np.maximum(disc, 0.0))
    inside = c < 0
    t = np.where(inside, -b + sq, -b - sq)
    hit = (disc >= 0) & (inside | (t > 0))
    q = o + t[:, None] * w
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(inside[:, None], -q, q) / sq[:, None]
    dist = np.where(hit, t, np.inf)
    g = np.where(hit[:, None], g, 0.0)
    return dist, hit, g
