"""Pins of the UDF oracle (Eq. 4) against facts that do not depend on it: for the analytic sphere
of radius r the true unsigned distance is | |x| - r |, which the minimum over a direction set
bounds from above and meets within the set's angular resolution (and exactly when the set holds
the direction to the nearest surface point); and a pure-Python loop over every (point, direction)
pair on a small network."""

import math

import numpy as np

from ddf_synth import fibonacci_directions, init_weights
from oracle import mlp as omlp
from oracle.sphere import sphere_ddf
from oracle.udf import udf


def _sphere_q(r):
    def q(o, w):
        d, hit, _ = sphere_ddf(o, w, r)
        return {"dist": np.where(hit, d, 0.0), "logit": np.where(hit, 1.0, -1.0)}
    return q


def test_sphere_udf_is_bounded_by_the_true_distance():
    r = 0.4
    rng = np.random.default_rng(1)
    P = rng.normal(size=(400, 3))
    P = (P / np.linalg.norm(P, axis=1, keepdims=True) * rng.uniform(0.05, 0.95, (400, 1))).astype(np.float32)
    D = fibonacci_directions(2000)
    u, arg, _ = udf(_sphere_q(r), P, D)
    true = np.abs(np.linalg.norm(P.astype(np.float64), axis=1) - r)
    assert (u >= true - 1e-7).all()
    # the set's largest angular gap: every direction has a set member within alpha
    probe = np.random.default_rng(2).normal(size=(20000, 3))
    probe /= np.linalg.norm(probe, axis=1, keepdims=True)
    alpha = np.arccos(np.clip((probe @ D.T.astype(np.float64)).max(1), -1, 1)).max()
    # outside: the chord to the sphere along a direction alpha off the centre exceeds |x| - r by
    # at most |x| (1 - cos alpha) + r (1 - cos beta) with sin beta = |x| sin alpha / r
    out = np.linalg.norm(P, axis=1) > r + 0.02
    x = np.linalg.norm(P[out].astype(np.float64), axis=1)
    sb = np.minimum(1.0, x * math.sin(alpha) / r)
    bound = x * (1 - math.cos(alpha)) + r * (1 - np.sqrt(1 - sb * sb))
    assert (u[out] - true[out] <= bound + 1e-9).all()
    assert (arg >= 0).all()


def test_sphere_udf_exact_when_the_set_holds_the_nearest_direction():
    r = 0.4
    P = np.array([[0.7, 0.0, 0.0], [0.0, -0.2, 0.0], [0.0, 0.0, 0.9]], np.float32)
    D = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float32)
    u, arg, _ = udf(_sphere_q(r), P, D)
    assert np.allclose(u, [0.3, 0.2, 0.5], rtol=0, atol=1e-7)
    assert arg.tolist() == [1, 3, 5]      # towards the centre outside, outwards inside


def test_udf_equals_a_loop_over_every_pair():
    F, W, L = 0, 32, 2
    blob = init_weights(F, W, L, seed=3)
    Pm = omlp.unpack(blob, F, W, L)
    rng = np.random.default_rng(4)
    P = rng.uniform(-0.5, 0.5, (7, 3)).astype(np.float32)
    D = fibonacci_directions(9)
    q = lambda o, w: omlp.query(Pm, o, w, F, with_normal=False)
    u, arg, gap = udf(q, P, D)
    for i in range(7):
        best, bk = math.inf, -1
        for k in range(9):
            y = omlp.query(Pm, P[i:i + 1], D[k:k + 1], F, with_normal=False)
            if y["logit"][0] > 0 and y["dist"][0] < best:
                best, bk = float(y["dist"][0]), k
        # one-row and batched products round differently in the last bits
        assert abs(u[i] - best) <= 1e-12 and (arg[i] == bk or gap[i] < 1e-12)
