"""A numpy model of the BF16 tensor-core arithmetic (test infrastructure).

It restates the network of Sec. 4.1 with BF16 rounding at the points where the tensor-core path
rounds: the encoded input, every hidden activation fed to the next GEMM, every weight matrix,
and every reverse-pass delta; products are accumulated exactly (the path accumulates in FP32).
At widths 128 and 256 the bias enters the accumulator as a BF16 hi / lo pair (split_bias).
The last hidden layer and the output head stay unrounded, as in the path. Comparing the GPU with
this model isolates kernel bugs from the inherent difference between a BF16-evaluated network
and the FP64 one (ReLU units whose sign flips under BF16 rounding change the gradient).
"""

import numpy as np
import torch

from oracle import mlp as omlp


def bf16(x):
    return torch.from_numpy(np.asarray(x, np.float64).astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def split_bias(b):
    """The bias as the width-128/256 kernels add it: one MMA of a ones column by the BF16 pair
    (bf16(b), bf16(b - bf16(b))), exact in the FP32 accumulator."""
    b32 = np.asarray(b, np.float64).astype(np.float32)
    hi = bf16(b32)
    lo = bf16((b32 - hi.astype(np.float32)).astype(np.float32))
    return hi + lo


def query_bf16(params, o, w, in_freqs, bias_in_mma=True):
    """bias_in_mma: the bias as split_bias gives it (widths 128 and 256); False: the FP32 bias
    added after the accumulation (width 512)."""
    X, dX = omlp.encode(o, w, in_freqs)
    L = len(params) - 1
    a = bf16(X)
    masks = []
    for l in range(L):
        Wl, b = params[l]
        z = a @ bf16(Wl).T + (split_bias(b) if bias_in_mma else b)
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


def train_grad_bf16(params, o, w, in_freqs, gy=None, dist_gt=None, hit_gt=None, snap=False, bias_in_mma=True,
                    loss_fn=None):
    """The reverse pass of the tensor-core training path with its BF16 rounding points: the
    encoded input, the hidden-layer weights, every hidden activation (the last one included:
    the output head reads it from memory), every delta; the output weights, y, G and the
    output-layer delta product in full precision. Returns (loss or None, [(dW, db)],
    d/d(o, w) (n, 6)).

    snap: round the encoded features to multiples of 2^-20, for inputs whose features are
    exactly 0 or +-1 (sin(k pi) evaluates to ~1e-16 in floating point, sinpi to exactly 0).
    loss_fn: y -> (loss, d loss / d y) in place of the two-output loss (the single-output heads)."""
    X, dX = omlp.encode(o, w, in_freqs)
    if snap:
        X = np.round(X * 2.0 ** 20) / 2.0 ** 20
    L = len(params) - 1
    a = bf16(X)
    acts, masks = [a], []
    for l in range(L):
        Wl, b = params[l]
        z = a @ bf16(Wl).T + (split_bias(b) if bias_in_mma else b)
        masks.append(z > 0)
        a = np.maximum(z, 0.0)
        if l < L - 1:
            a = bf16(a)
            acts.append(a)
    Wo, bo = params[L]
    aL = bf16(a)
    y = aL @ Wo.T + bo
    loss = None
    if gy is None and loss_fn is not None:
        loss, gy = loss_fn(y)
    elif gy is None:
        loss, gy = omlp.loss_and_output_grad(y, dist_gt, hit_gt)
    grads = [None] * (L + 1)
    grads[L] = (gy.T @ aL, gy.sum(0))
    d = bf16((gy @ Wo) * masks[L - 1])
    for l in range(L - 1, -1, -1):
        grads[l] = (d.T @ acts[l], d.sum(0))
        if l > 0:
            d = bf16((d @ bf16(params[l][0])) * masks[l - 1])
    gX = d @ bf16(params[0][0])
    gf = gX * dX
    g = np.zeros((X.shape[0], 6))
    for f in range(X.shape[1]):
        g[:, f % 6] += gf[:, f]
    return loss, grads, g
