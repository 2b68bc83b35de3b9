"""Pins of the oracle's Philox4x32-10 against the generator authors' published
known-answer vectors (SC'11), and of its uniform mapping."""

import os

import numpy as np

from oracle.philox import philox4x32_10, uniform24, path_uniforms

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(x, 16) for x in line.split()])
    return np.array(rows, dtype=np.uint64)


def test_known_answer_vectors():
    kat = _kat()
    assert kat.shape == (3, 10)
    for row in kat:
        out = philox4x32_10(row[None, 0:4].astype(np.uint32), row[4:6].astype(np.uint32))
        assert out[0].tolist() == row[6:10].astype(np.uint32).tolist()


def test_vectorised_matches_rowwise():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(64, 2), dtype=np.uint64).astype(np.uint32)
    batch = philox4x32_10(ctr, key)
    for i in range(64):
        assert (philox4x32_10(ctr[i:i + 1], key[i]) == batch[i:i + 1]).all()


def test_uniform24_range_and_exactness():
    x = np.array([0, 255, 256, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    u = uniform24(x)
    assert u[0] == 0.0 and u[1] == 0.0
    assert u[2] == 2.0 ** -24
    assert u[3] == 1.0 - 2.0 ** -24
    assert u[4] == 0.5
    # exactly representable in float32
    assert (u.astype(np.float32).astype(np.float64) == u).all()


def test_path_stream_layout():
    pid = np.array([0, 1, (1 << 32) + 5], dtype=np.uint64)
    u = path_uniforms(0x0000000100000002, pid, 3)
    ctr = np.array([[0, 0, 3, 0], [1, 0, 3, 0], [5, 1, 3, 0]], dtype=np.uint32)
    ref = uniform24(philox4x32_10(ctr, np.array([2, 1], dtype=np.uint32)))
    assert (u == ref).all()
    # streams of different bounces differ
    assert not np.array_equal(path_uniforms(1, pid, 0), path_uniforms(1, pid, 1))
