"""FP64 DDF network: forward, input gradient (surface normal), parameter gradient,
training loss and Adam. Test infrastructure only (see the package docstring).

Network (Sec. 4.1, MLP_w: (x, theta) -> field value; sizes of Sec. 5.1): an oriented
point is encoded, passed through L hidden layers z_l = W_l a_{l-1} + b_l,
a_l = ReLU(z_l), and an output layer y = W_out a_L + b_out with two outputs:
y_0 = distance, y_1 = hit logit (hit <=> y_1 > 0). The two-output head, the 6-D input
(origin + unit direction instead of two angles, the angle form of Eq. 1 being only a
parameterisation of the same direction) and the Fourier encoding are readings of this
implementation; the paper's single clamped output is the head of ``oracle.head``.

Encoding (reading): v = (o_x, o_y, o_z, w_x, w_y, w_z); with F = in_freqs (even),
gamma(v) = [v_0..v_5, then for k = 0 .. F/2 - 1: sin(2^k pi v_j) for j = 0..5,
cos(2^k pi v_j) for j = 0..5], i.e. E = 6 + 6F features (F = 12 -> 78, F = 16 -> 102).

ReLU'(0) := 0.

Normal (Eq. 3, Sec. 4.2): g = d y_0 / d o, the gradient of the distance output w.r.t.
the query origin (taken at the query origin, as the paper's autodiff listing does);
n = kappa g / |g| with kappa in {-1, +1} chosen so that n . w < 0 (kappa = +1 when
g . w == 0); n = -w when |g| == 0.

Loss (reading of the training objective for the two-output head): mean over rays with
hit_gt = 1 of |y_0 - dist_gt| (0 if there are none) plus the mean over all rays of the
binary cross-entropy with logits, max(z, 0) - z*h + log(1 + exp(-|z|)). The L1
subgradient at 0 is 0.

Adam (Kingma & Ba): m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
w <- w - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""

from __future__ import annotations

import numpy as np


def unpack(blob, in_freqs: int, width: int, hidden_layers: int):
    """Flat [W_1, b_1, ..., W_out, b_out] blob -> list of float64 (W, b)."""
    E = 6 + 6 * in_freqs
    shapes = [(width, E)] + [(width, width)] * (hidden_layers - 1) + [(2, width)]
    blob = np.asarray(blob, dtype=np.float64)
    out, off = [], 0
    for o, i in shapes:
        W = blob[off:off + o * i].reshape(o, i)
        off += o * i
        b = blob[off:off + o]
        off += o
        out.append((W, b))
    if off != blob.size:
        raise ValueError("weight blob size mismatch")
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def encode(o, w, in_freqs: int):
    """gamma(v) and the per-feature derivative d gamma_f / d v_{j(f)} (both (n, E))."""
    v = np.concatenate([np.asarray(o, np.float64), np.asarray(w, np.float64)], axis=1)
    feats = [v]
    dfeat = [np.ones_like(v)]
    for k in range(in_freqs // 2):
        f = (2.0 ** k) * np.pi
        feats.append(np.sin(f * v))
        dfeat.append(f * np.cos(f * v))
        feats.append(np.cos(f * v))
        dfeat.append(-f * np.sin(f * v))
    return np.concatenate(feats, axis=1), np.concatenate(dfeat, axis=1)


def forward(params, X):
    """X: (n, E) encoded inputs. Returns y (n, 2) and the per-layer pre-activations z_l
    and activations a_l (a_0 = X)."""
    a = X
    acts, pres = [a], []
    for W, b in params[:-1]:
        z = a @ W.T + b
        a = np.maximum(z, 0.0)
        pres.append(z)
        acts.append(a)
    Wo, bo = params[-1]
    y = a @ Wo.T + bo
    return y, pres, acts


def backward(params, pres, acts, gy):
    """Reverse pass for output cotangent gy (n, 2): returns (param grads list of (dW, db),
    gX (n, E) = d/dX of sum(gy * y))."""
    grads = [None] * len(params)
    Wo, _ = params[-1]
    grads[-1] = (gy.T @ acts[-1], gy.sum(0))
    d = (gy @ Wo) * (pres[-1] > 0)
    for l in range(len(params) - 2, -1, -1):
        W, _ = params[l]
        grads[l] = (d.T @ acts[l], d.sum(0))
        g_prev = d @ W
        if l > 0:
            d = g_prev * (pres[l - 1] > 0)
    return grads, g_prev


def input_gradient(params, o, w, in_freqs: int):
    """d y_0 / d (o, w): (n, 6)."""
    X, dX = encode(o, w, in_freqs)
    y, pres, acts = forward(params, X)
    gy = np.zeros_like(y)
    gy[:, 0] = 1.0
    _, gX = backward(params, pres, acts, gy)
    gf = gX * dX
    n6 = np.zeros((X.shape[0], 6))
    E = X.shape[1]
    for f in range(E):
        n6[:, f % 6] += gf[:, f]
    return y, n6


def normal_from_gradient(g_o, w):
    """Eq. 3 with kappa chosen so that n . w < 0; n = -w when the gradient vanishes."""
    g_o = np.asarray(g_o, np.float64)
    w = np.asarray(w, np.float64)
    nrm = np.sqrt(np.sum(g_o * g_o, axis=1, keepdims=True))
    n = np.where(nrm > 0, g_o / np.where(nrm > 0, nrm, 1.0), -w)
    flip = np.sum(n * w, axis=1) > 0
    n[flip] = -n[flip]
    return n


def query(params, o, w, in_freqs: int, with_normal: bool = True):
    """The DDF query: distance, logit, hit and (optionally) the Eq. 3 normal."""
    if with_normal:
        y, g = input_gradient(params, o, w, in_freqs)
        n = normal_from_gradient(g[:, :3], w)
    else:
        X, _ = encode(o, w, in_freqs)
        y, _, _ = forward(params, X)
        g, n = None, None
    return {"dist": y[:, 0], "logit": y[:, 1], "hit": y[:, 1] > 0, "grad": g, "normal": n}


def loss_and_output_grad(y, dist_gt, hit_gt):
    """Training loss and d loss / d y (n, 2)."""
    d, z = y[:, 0], y[:, 1]
    h = np.asarray(hit_gt).astype(np.float64)
    n = y.shape[0]
    n_hit = int(np.sum(h > 0))
    gy = np.zeros_like(y)
    l1 = 0.0
    if n_hit > 0:
        m = h > 0
        diff = d[m] - np.asarray(dist_gt, np.float64)[m]
        l1 = np.sum(np.abs(diff)) / n_hit
        gy[m, 0] = np.sign(diff) / n_hit
    bce = np.mean(np.maximum(z, 0.0) - z * h + np.log1p(np.exp(-np.abs(z))))
    gy[:, 1] = (1.0 / (1.0 + np.exp(-z)) - h) / n
    return l1 + bce, gy


def param_gradient(params, o, w, in_freqs, dist_gt, hit_gt):
    X, _ = encode(o, w, in_freqs)
    y, pres, acts = forward(params, X)
    L, gy = loss_and_output_grad(y, dist_gt, hit_gt)
    grads, _ = backward(params, pres, acts, gy)
    return L, grads, y


def adam_update(wts, g, m, v, step: int, lr: float, b1: float, b2: float, eps: float):
    """One Adam step on flat float64 arrays; returns (w, m, v). `step` counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return wts - lr * mh / (np.sqrt(vh) + eps), m, v
