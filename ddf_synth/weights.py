"""Seeded DDF network weights in the flat float32 layout the C ABI takes.

Layout: [W_1, b_1, W_2, b_2, ..., W_L, b_L, W_out, b_out], each W row-major [out][in]
(the nn.Linear convention). Hidden layers have `width` units; the first takes the encoded
input of E = 6 + 6 * in_freqs features; the output layer has 2 units (distance, hit logit).
"""

from __future__ import annotations

import numpy as np


def encoded_width(in_freqs: int) -> int:
    return 6 + 6 * in_freqs


def ddf_arch_sizes(in_freqs: int, width: int, hidden_layers: int):
    """List of (out, in) shapes of the L hidden layers and the output layer."""
    E = encoded_width(in_freqs)
    shapes = [(width, E)] + [(width, width)] * (hidden_layers - 1) + [(2, width)]
    return shapes


def n_params(in_freqs: int, width: int, hidden_layers: int) -> int:
    return sum(o * i + o for o, i in ddf_arch_sizes(in_freqs, width, hidden_layers))


def init_weights(in_freqs: int, width: int, hidden_layers: int, seed: int, bias_scale: float = 0.1,
                 zero_bias: bool = False) -> np.ndarray:
    """Glorot-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)); biases
    U(-bias_scale, bias_scale) (all zero when zero_bias). Returns the flat float32 blob."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in ddf_arch_sizes(in_freqs, width, hidden_layers):
        a = np.sqrt(6.0 / (i + o))
        parts.append(rng.uniform(-a, a, size=(o, i)).ravel())
        if zero_bias:
            parts.append(np.zeros(o))
        else:
            parts.append(rng.uniform(-bias_scale, bias_scale, size=o))
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


def split_weights(blob: np.ndarray, in_freqs: int, width: int, hidden_layers: int):
    """Views [(W, b), ...] into a flat blob (any float dtype)."""
    out = []
    off = 0
    for o, i in ddf_arch_sizes(in_freqs, width, hidden_layers):
        W = blob[off:off + o * i].reshape(o, i)
        off += o * i
        b = blob[off:off + o]
        off += o
        out.append((W, b))
    assert off == blob.size, (off, blob.size)
    return out
