"""bench.py's roofline arithmetic on the CPU: the algorithmic flops per query and per normal of the
headline network (written out from the layer sizes), the per-row DRAM bytes of the query kernels
against the algorithmic ray bytes, and the traffic of a render from its rows per bounce."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_flops_of_the_headline_network():
    E, W, L = 6 + 6 * 12, 256, 8
    # forward: E x W, then L - 1 hidden W x W layers, then the 2-unit head; 2 flops per MAC
    assert bench.fwd_flops(E, W, L) == 2 * (78 * 256 + 7 * 256 * 256 + 2 * 256) == 958464
    # reverse for a normal: L - 1 W x W layers and the W x E first layer
    assert bench.bwd_flops(E, W, L) == 2 * (7 * 256 * 256 + 256 * 78) == 957440


def test_query_dram_bytes_stay_within_the_ray_bytes():
    # forward: 24 B of ray in, 9 B out (distance, logit, hit) and a 4 B hit-list entry at most
    assert bench.QUERY_DRAM_BYTES_PER_FWD_ROW <= 24 + 9 + 4
    # normals: the 4 B list entry, the 24 B ray, the 12 B normal
    assert bench.QUERY_DRAM_BYTES_PER_NRM_ROW <= 4 + 24 + 12
    assert bench.QUERY_DRAM_BYTES_PER_FWD_ROW >= 24   # the rays are read once


def test_render_traffic_from_rows_per_bounce():
    stats = [16777216, 2530338, 374863, 59172]
    f, n = bench.QUERY_DRAM_BYTES_PER_FWD_ROW, bench.QUERY_DRAM_BYTES_PER_NRM_ROW
    want = (f * sum(stats) + n * (2530338 + 374863 + 59172)) / 4
    assert bench.query_traffic_per_bounce(stats, 4) == pytest.approx(want)
    assert bench.query_traffic_per_bounce(stats, 4) == pytest.approx(173.9e6, rel=1e-3)


def test_whole_job_rate_counts_every_rank():
    # 2 ranks x 3 steps x 100 units in 15 ms
    assert bench.whole_job_rate(100, 2, 3, 15.0) == pytest.approx(600 / 0.015)
