"""A numpy/torch model of the FP8 E4M3 tensor-core arithmetic (test infrastructure).

It restates the network of Sec. 4.1 with the FP8 path's quantisation, given the path's static
activation scales s_a [L][W] (read back from the library: they come from a calibration pass):
hidden layer l's weights are folded with its input scales, W'[n, k] = W[n, k] s_a[l][k], scaled
per output channel by s_w[n] and rounded to E4M3. For l < L - 1 the weight scale is tied to the
next layer's input scale of the same unit, s_w[n] = mu_l s_a[l + 1][n], with one mu_l per layer
chosen so that the largest weight code is 448; the last hidden layer uses max_k |W'[n, k]| / 448.
The layer input is rounded to E4M3 as a[k] / s_a[l][k] (layer 0: a[k] 448); the products
accumulate exactly and z = acc s_w + b. The last hidden layer's output and the output head stay
in floating point.
"""

import numpy as np
import torch

from oracle import mlp as omlp


def e4m3(x):
    """Round to E4M3 with saturation at +-448 (the conversion the kernels use)."""
    t = torch.from_numpy(np.clip(np.asarray(x, np.float64).astype(np.float32), -448.0, 448.0))
    return t.to(torch.float8_e4m3fn).to(torch.float64).numpy()


def f32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def query_fp8(params, o, w, in_freqs, sa):
    """sa: float32 [L, width] static activation scales; layer 0 uses sa[0][:E]."""
    X, _ = omlp.encode(o, w, in_freqs)
    L = len(params) - 1
    a = X
    for l in range(L):
        Wl, b = params[l]
        s = np.asarray(sa[l][: Wl.shape[1]], np.float64)
        Wp = f32(f32(Wl) * s[None, :])
        r = np.abs(Wp).max(axis=1)
        if l < L - 1:
            # weight scale tied to the next layer's input scale: s_w = mu s_a', one mu per layer
            nxt = np.asarray(sa[l + 1][: Wl.shape[0]], np.float64)
            mu = f32((r / f32(448.0 * nxt)).max())
            mu = mu if mu > 0 else 1.0
            sw = f32(mu * nxt)
        else:
            sw = f32(r / 448.0)
            sw[sw == 0] = 1.0
        Wq = e4m3(Wp * f32(1.0 / sw)[:, None])
        inv = np.full_like(s, 448.0) if l == 0 else f32(1.0 / s)
        aq = e4m3(f32(a) * inv[None, :])
        z = (aq @ Wq.T) * sw[None, :] + b
        a = np.maximum(z, 0.0)
    Wo, bo = params[L]
    y = a @ Wo.T + bo
    return {"dist": y[:, 0], "logit": y[:, 1], "hit": y[:, 1] > 0}


def calibration_bound(params, o, w, in_freqs):
    """Column maxima of |a_l| (FP64 forward) for l = 1 .. L-1 on the given rays: [L, width],
    row 0 zero. The static scales must cover them: 448 s_a / 2 is about this maximum."""
    X, _ = omlp.encode(o, w, in_freqs)
    L = len(params) - 1
    W = params[0][0].shape[0]
    out = np.zeros((L, W))
    a = X
    for l in range(L - 1):
        Wl, b = params[l]
        a = np.maximum(a @ Wl.T + b, 0.0)
        out[l + 1] = np.abs(a).max(axis=0)
    return out
