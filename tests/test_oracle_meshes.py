"""Pins of the synthetic meshes the workloads use (counts, topology, placement)."""

import numpy as np
import pytest

from ddf_synth import icosphere, torus, torus_knot, mesh_euler_characteristic


def _signed_volume(V, F):
    V = V.astype(np.float64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0)


@pytest.mark.parametrize("level,nt", [(0, 20), (1, 80), (2, 320), (3, 1280)])
def test_icosphere_counts_topology(level, nt):
    V, F = icosphere(level, 0.5)
    assert F.shape == (nt, 3)
    assert V.shape[0] == 10 * 4 ** level + 2
    assert mesh_euler_characteristic(V, F) == 2
    r = np.linalg.norm(V.astype(np.float64), axis=1)
    assert np.allclose(r, 0.5, rtol=0, atol=1e-7)
    assert _signed_volume(V, F) > 0          # outward winding
    assert _signed_volume(V, F) < 4 / 3 * np.pi * 0.125


def test_torus_topology():
    V, F = torus(0.6, 0.25, 32, 16)
    assert F.shape == (1024, 3)
    assert mesh_euler_characteristic(V, F) == 0
    vol = _signed_volume(V, F)
    exact = 2 * np.pi ** 2 * 0.6 * 0.25 ** 2
    assert 0.9 * exact < vol < exact          # inscribed polyhedron, outward


@pytest.mark.parametrize("ns,nr,nt", [(256, 16, 8192), (1024, 64, 131072)])
def test_torus_knot(ns, nr, nt):
    V, F = torus_knot(3, 2, 0.08, ns, nr)
    assert F.shape == (nt, 3)
    assert mesh_euler_characteristic(V, F) == 0
    assert np.linalg.norm(V.astype(np.float64), axis=1).max() <= 0.95 + 1e-6
    vol = _signed_volume(V, F)
    assert vol > 0
