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


def test_fibonacci_directions_cover_the_sphere_evenly():
    """The UDF's default direction set: unit float32 vectors whose every spherical cap of a given
    area holds about its share (the lattice's discrepancy is small), and whose largest angular gap
    shrinks like 1 / sqrt(k)."""
    from ddf_synth import fibonacci_directions
    for k in (64, 256, 1024):
        d = fibonacci_directions(k).astype(np.float64)
        assert d.shape == (k, 3) and np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-6
        assert np.abs(d.mean(0)).max() < 2.0 / k + 1e-3
        probe = np.random.default_rng(k).normal(size=(4000, 3))
        probe /= np.linalg.norm(probe, axis=1, keepdims=True)
        gap = np.arccos(np.clip((probe @ d.T).max(1), -1, 1)).max()
        assert gap < 3.0 / np.sqrt(k)
        # caps of half-angle 60 degrees hold a quarter of the sphere
        frac = ((probe[:50] @ d.T) > 0.5).mean(1)
        assert np.abs(frac - 0.25).max() < 0.05 + 4.0 / np.sqrt(k)
