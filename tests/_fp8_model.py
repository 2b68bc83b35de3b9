"""A numpy/torch model of the FP8 E4M3 tensor-core arithmetic (test infrastructure).

It restates the network of Sec. 4.1 with the FP8 path's quantisation: every hidden layer's
weights scaled per output channel by max |W[n, :]| / 448 and rounded to E4M3, every layer input
row scaled by max |a[r, :]| / 448 and rounded to E4M3, exact accumulation, then
z = acc * s_a * s_w + b; the last hidden layer and the output head stay in floating point.
"""

import numpy as np
import torch

from oracle import mlp as omlp


def e4m3(x):
    t = torch.from_numpy(np.asarray(x, np.float64).astype(np.float32))
    return t.to(torch.float8_e4m3fn).to(torch.float64).numpy()


def query_fp8(params, o, w, in_freqs):
    X, _ = omlp.encode(o, w, in_freqs)
    L = len(params) - 1
    a = X
    for l in range(L):
        Wl, b = params[l]
        sw = np.abs(Wl).max(axis=1) / 448.0
        sw[sw == 0] = 1.0
        Wq = e4m3(Wl / sw[:, None])
        sa = np.abs(a).max(axis=1) / 448.0
        sa[sa == 0] = 1.0
        aq = e4m3(a / sa[:, None])
        z = (aq @ Wq.T) * sa[:, None] * sw[None, :] + b
        a = np.maximum(z, 0.0)
    Wo, bo = params[L]
    y = a @ Wo.T + bo
    return {"dist": y[:, 0], "logit": y[:, 1], "hit": y[:, 1] > 0}
