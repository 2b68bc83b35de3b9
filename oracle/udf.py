"""The unsigned distance field recovered from a DDF (Eq. 4): UDF(x) = min over directions theta
of phi(x, theta). Test infrastructure only (see the package docstring).

Readings: the minimum runs over a given finite set of unit directions (the paper's minimum over
all directions is its limit as the set fills the sphere), and only over directions whose ray hits
(the field value of a miss is infinite, Sec. 4.1); +inf if none hits. The minimising direction
is the lowest index among equal distances.
"""

from __future__ import annotations

import numpy as np


def udf(query_fn, points, dirs):
    """query_fn(o, w) -> dict(dist, logit) in float64. Returns (udf (n,), argmin (n,), gap (n,)),
    gap = the second smallest hit distance minus the smallest (+inf with fewer than two hits),
    which says how far the argmin decision is from a tie."""
    P = np.asarray(points, np.float32)
    D = np.asarray(dirs, np.float32)
    n, k = P.shape[0], D.shape[0]
    o = np.repeat(P, k, axis=0)
    w = np.tile(D, (n, 1))
    res = query_fn(o, w)
    d = np.where(np.asarray(res["logit"]) > 0, np.asarray(res["dist"], np.float64), np.inf).reshape(n, k)
    arg = np.argmin(d, axis=1)                       # first minimum: the lowest index on ties
    best = d[np.arange(n), arg]
    arg = np.where(np.isfinite(best), arg, -1)
    srt = np.sort(d, axis=1)
    gap = srt[:, 1] - srt[:, 0] if k > 1 else np.full(n, np.inf)
    return best, arg, gap
