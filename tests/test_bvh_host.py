"""The labeller's bounding-volume hierarchy, built and checked on the host (ddf_bvh_selfcheck, no
GPU): every face in exactly one leaf, padded leaf boxes holding their faces, child boxes inside
their parents', every node reached once, depth within the traversal stack, on ordinary meshes
and on the awkward ones (duplicated faces, coincident and zero-area faces, one face, a flat
grid)."""

import ctypes

import numpy as np
import pytest

from ddf_synth import icosphere, torus_knot
from tests._helpers import ensure_built


def _check(V, T):
    ensure_built()
    from paper_2306_16142_gb300 import _abi
    lib = _abi.load()
    V = np.ascontiguousarray(V, np.float32)
    T = np.ascontiguousarray(T, np.int32)
    out = (ctypes.c_int64 * 4)()
    rc = lib.ddf_bvh_selfcheck(V.ctypes.data_as(ctypes.c_void_p), V.shape[0], T.ctypes.data_as(ctypes.c_void_p),
                               T.shape[0], out)
    return rc, lib.ddf_last_error().decode(), list(out)


def _grid(n):
    x, y = np.meshgrid(np.linspace(-0.9, 0.9, n + 1), np.linspace(-0.9, 0.9, n + 1))
    V = np.stack([x.ravel(), y.ravel(), np.zeros(x.size)], 1)
    idx = np.arange((n + 1) * (n + 1)).reshape(n + 1, n + 1)
    a, b, c, d = idx[:-1, :-1].ravel(), idx[:-1, 1:].ravel(), idx[1:, 1:].ravel(), idx[1:, :-1].ravel()
    return V, np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)])


CASES = {
    "icosphere": lambda: icosphere(3, 0.5),
    "knot 8192": lambda: torus_knot(3, 2, 0.08, 256, 16),
    "knot 131072": lambda: torus_knot(3, 2, 0.08, 1024, 64),
    "flat grid": lambda: _grid(64),
    "duplicated faces": lambda: (lambda V, T: (V, np.concatenate([T, T[::-1], T])))(*icosphere(2, 0.5)),
    "one face": lambda: (np.float32([[0, 0, 0], [1, 0, 0], [0, 1, 0]]), np.int32([[0, 1, 2]])),
    "two faces": lambda: (np.float32([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]]), np.int32([[0, 1, 2], [1, 3, 2]])),
    "coincident faces": lambda: (np.float32([[0, 0, 0], [1, 0, 0], [0, 1, 0]]), np.zeros((500, 3), np.int32) + [0, 1, 2]),
    "zero-area faces": lambda: (np.float32([[0, 0, 0], [0.5, 0.5, 0.5], [1, 1, 1], [0.2, 0.2, 0.2]]),
                                np.int32([[0, 1, 2], [1, 2, 3], [0, 3, 2]] * 40)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_hierarchy_invariants(name):
    V, T = CASES[name]()
    rc, err, (nodes, depth, leaves, largest) = _check(V, T)
    assert rc == 0, err
    assert nodes >= 1 and 0 <= depth <= 56 and leaves >= 1
    if name in ("icosphere", "knot 8192", "knot 131072", "flat grid"):
        assert largest <= 8 and depth <= 40
        # a sensible tree: about one node per two to four faces
        assert T.shape[0] / 8 <= nodes <= T.shape[0]


def test_bad_meshes_are_rejected():
    V, T = icosphere(1, 0.5)
    T2 = T.copy()
    T2[3, 1] = V.shape[0]                      # out of range
    rc, err, _ = _check(V, T2)
    assert rc != 0 and "references vertex" in err
