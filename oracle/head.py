"""The paper's own network head and training variant (Sec. 4.1 and Sec. 5.1): a single field
value y~ trained with the clamp loss of Eq. 7 or the squish loss of Eq. 5, and weight-normalised
hidden layers. Test infrastructure only (see the package docstring).

Readings (the paper is silent or garbled):

* Single output. A ray hits <=> y~ < delta: the clamp's half-width delta is the distance up to
  which the field is learnt, the paper's "draw distance". A two-output network realises this
  head with a derived second row, W_out[1] = -W_out[0] and b_out[1] = delta - b_out[0], so that
  its logit is delta - y~ and "logit > 0" is the same test.
* Target. y is the labelled distance of a ray that hits and +inf for one that misses (the
  infinite field value of Sec. 4.1); clamp(+inf, delta) = delta and tanh(+inf) = 1.
* Losses are means over all rays. Eq. 5 as printed is a signed difference, which is not a loss;
  the reading is its absolute value, |sigma(y) - sigma(y~)| with sigma = tanh.
* Derivatives. clamp(x, delta) has derivative 1 on the closed interval [-delta, delta] and 0
  outside; |x| has sign(x), 0 at 0.
* Weight normalisation (Salimans and Kingma, 2016) on every hidden layer ("8 weight-normalized
  hidden layers"), per output row: W[r, :] = g[r] v[r, :] / |v[r, :]|; biases and the output
  layer stay plain parameters. Switching it on sets v = W and g[r] = |W[r, :]|.
"""

from __future__ import annotations

import numpy as np


def derive_single_head(params, delta: float):
    """The two-output parameter list whose logit is delta - y~ (row 1 derived from row 0)."""
    Wo, bo = params[-1]
    Wo = np.array(Wo, np.float64)
    bo = np.array(bo, np.float64)
    Wo[1] = -Wo[0]
    bo[1] = delta - bo[0]
    return list(params[:-1]) + [(Wo, bo)]


def _target(dist_gt, hit_gt):
    h = np.asarray(hit_gt) > 0
    return np.where(h, np.asarray(dist_gt, np.float64), np.inf)


def clamp_loss_and_output_grad(y, dist_gt, hit_gt, delta: float):
    """Eq. 7: mean |clamp(y_gt, delta) - clamp(y~, delta)| and d loss / d y (n, 2) (the logit
    row gets none)."""
    d = y[:, 0]
    n = y.shape[0]
    cy = np.minimum(delta, np.maximum(-delta, _target(dist_gt, hit_gt)))
    cd = np.minimum(delta, np.maximum(-delta, d))
    diff = cd - cy
    gy = np.zeros_like(y)
    inside = (d >= -delta) & (d <= delta)
    gy[:, 0] = np.sign(diff) * inside / n
    return float(np.mean(np.abs(diff))), gy


def squish_loss_and_output_grad(y, dist_gt, hit_gt):
    """Eq. 5 (with the absolute value): mean |tanh(y_gt) - tanh(y~)| and d loss / d y (n, 2)."""
    d = y[:, 0]
    n = y.shape[0]
    ty = np.tanh(_target(dist_gt, hit_gt))
    td = np.tanh(d)
    diff = td - ty
    gy = np.zeros_like(y)
    gy[:, 0] = np.sign(diff) * (1.0 - td * td) / n
    return float(np.mean(np.abs(diff))), gy


def wn_init(W):
    """(v, g) of a weight matrix: v = W, g = row norms."""
    W = np.asarray(W, np.float64)
    return W.copy(), np.linalg.norm(W, axis=1)


def wn_fold(v, g):
    """W = g v / |v| per row."""
    v = np.asarray(v, np.float64)
    return (np.asarray(g, np.float64) / np.linalg.norm(v, axis=1))[:, None] * v


def wn_grad(v, g, dW):
    """Gradients of (v, g) from the gradient dW of the folded weight: with u = v / |v|,
    dg = dW . u and dv = (g / |v|) (dW - dg u), per row."""
    v = np.asarray(v, np.float64)
    nv = np.linalg.norm(v, axis=1)
    u = v / nv[:, None]
    dg = np.sum(dW * u, axis=1)
    dv = (np.asarray(g, np.float64) / nv)[:, None] * (dW - dg[:, None] * u)
    return dv, dg
