"""Shared test helpers: building/loading the library, seeded workloads, tolerances."""

from __future__ import annotations

import numpy as np

# FP32 query tolerance: |dy| <= 1e-5 * max(|y64|, 1) (relative, floored at 1 in the unit scene).
FP32_REL = 1e-5
# Hit decisions are compared only where the oracle's logit is at least this far from 0.
LOGIT_MARGIN = 1e-4
# BF16 distance tolerance (absolute, unit scene).
BF16_ABS = 2e-2

_built = False


def ensure_built():
    global _built
    if not _built:
        from paper_2306_16142_gb300 import build
        build.build()
        _built = True


# name: (in_freqs, width, hidden_layers, seed, zero_bias)
NETS = {
    "tiny_6x64x4": (0, 64, 4, 0, True),            # the tiny plain-method network
    "train_78x256x8": (12, 256, 8, 2, False),       # training / single-object render shape
    "large_102x512x8": (16, 512, 8, 5, False),      # large-render shape
}


def net_weights(name):
    from ddf_synth import init_weights
    F, W, L, seed, zb = NETS[name]
    return init_weights(F, W, L, seed=seed, zero_bias=zb)


def rays_in_ball(n, seed):
    """Origins uniform in the unit ball's shell/interior mix, unit directions."""
    rng = np.random.default_rng(seed)
    o = rng.normal(size=(n, 3))
    o /= np.linalg.norm(o, axis=1, keepdims=True)
    o *= rng.uniform(0.2, 1.0, size=(n, 1))
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    return o.astype(np.float32), w.astype(np.float32)


def fp32_close(y32, y64, rel=FP32_REL):
    y32 = np.asarray(y32, np.float64)
    y64 = np.asarray(y64, np.float64)
    return np.abs(y32 - y64) <= rel * np.maximum(np.abs(y64), 1.0)
