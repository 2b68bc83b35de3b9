"""A numpy model of the BF16 tensor-core arithmetic (test infrastructure).

It restates the network of Sec. 4.1 with BF16 rounding at the points where the tensor-core path
rounds: the encoded input, every hidden activation fed to the next GEMM, every weight matrix,
and every reverse-pass delta; products are accumulated exactly (the path accumulates in FP32).
The last hidden layer and the output head stay unrounded, as in the path. Comparing the GPU with
this model isolates kernel bugs from the inherent difference between a BF16-evaluated network
and the FP64 one (ReLU units whose sign flips under BF16 rounding change the gradient).
"""

import numpy as np
import torch

from oracle import mlp as omlp


def bf16(x):
    return torch.from_numpy(np.asarray(x, np.float64).astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def query_bf16(params, o, w, in_freqs):
    X, dX = omlp.encode(o, w, in_freqs)
    L = len(params) - 1
    a = bf16(X)
    masks = []
    for l in range(L):
        Wl, b = params[l]
        z = a @ bf16(Wl).T + b
        masks.append(z > 0)
        a = np.maximum(z, 0.0)
        if l < L - 1:
            a = bf16(a)
    Wo, bo = params[L]
    y = a @ Wo.T + bo
    d = bf16(np.where(masks[L - 1], Wo[0][None, :], 0.0))
    for l in range(L - 1, 0, -1):
        d = bf16((d @ bf16(params[l][0])) * masks[l - 1])
    gX = d @ bf16(params[0][0])
    gf = gX * dX
    g = np.zeros((X.shape[0], 6))
    for f in range(X.shape[1]):
        g[:, f % 6] += gf[:, f]
    return {"dist": y[:, 0], "logit": y[:, 1], "hit": y[:, 1] > 0, "grad": g,
            "normal": omlp.normal_from_gradient(g[:, :3], w)}
