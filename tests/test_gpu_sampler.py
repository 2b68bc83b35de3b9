"""GPU surface-marching sampler (Sec. 5.2, Eqs. 8-12, odd-even inside test) against the FP64
oracle (oracle/sampler.py): the same samples, bit for bit (keys, hit flags, float32 coordinates
and distances), on a convex icosphere, a non-convex pair of spheres and a torus knot; the cap and
empty cases; determinism."""

import numpy as np
import pytest
import torch

from ddf_synth import icosphere, torus_knot
from oracle import sampler as S
from tests._helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


def _two_spheres():
    Va, Ta = icosphere(2, 0.3)
    Vb = Va.copy()
    Va = Va + np.float32([-0.45, 0.0, 0.0])
    Vb = Vb + np.float32([0.45, 0.0, 0.0])
    return np.concatenate([Va, Vb]).astype(np.float32), np.concatenate([Ta, Ta + Va.shape[0]]).astype(np.int32)


CASES = {
    "icosphere": (lambda: icosphere(2, 0.5), (2, 4, 4, 1e-4, 11)),
    "two_spheres": (_two_spheres, (1, 6, 5, 1e-4, 3)),
    "knot": (lambda: torus_knot(3, 2, 0.08, 64, 8), (1, 3, 3, 2e-4, 7)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_sampler_matches_oracle_bit_for_bit(P, name):
    make, (s_fc, s_dr, s_p, eps, seed) = CASES[name]
    V, T = make()
    mesh = P.DDFMesh(V, T)
    g = mesh.sample_surface(s_fc, s_dr, s_p, eps, seed)
    torch.cuda.synchronize()
    r = S.sample_surface(V, T, s_fc, s_dr, s_p, eps, seed)
    n = r["key"].shape[0]
    print(f"{name}: {n} samples from {T.shape[0] * s_fc * s_dr} rays; kinds",
          np.bincount(r["key"] % 4, minlength=4))
    assert n > 0 and g["count"] == n
    gk = g["key"].cpu().numpy()
    assert np.array_equal(gk, r["key"])
    assert np.array_equal(g["hit"].cpu().numpy(), r["hit"])
    assert np.array_equal(g["dist"].cpu().numpy(), r["dist"])
    go, gw = g["o"].cpu().numpy(), g["w"].cpu().numpy()
    bad = np.nonzero(np.any(go != r["o"], axis=1) | np.any(gw != r["w"], axis=1))[0]
    assert bad.size == 0, (bad[:5], go[bad[:3]], r["o"][bad[:3]], gw[bad[:3]], r["w"][bad[:3]])


def test_sampler_cap_empty_and_determinism(P):
    V, T = _two_spheres()
    mesh = P.DDFMesh(V, T)
    full = mesh.sample_surface(1, 2, 3, 1e-4, 5)
    n = full["count"]
    assert n > 100
    part = mesh.sample_surface(1, 2, 3, 1e-4, 5, cap=n // 3)
    assert part["count"] == n and part["key"].shape[0] == n // 3
    assert torch.equal(part["key"], full["key"][: n // 3])
    assert torch.equal(part["o"], full["o"][: n // 3])
    again = mesh.sample_surface(1, 2, 3, 1e-4, 5)
    for k in ("o", "w", "dist", "hit", "key"):
        assert torch.equal(again[k], full[k])
    assert mesh.sample_surface(1, 2, 0, 1e-4, 5)["count"] == 0
    assert mesh.sample_surface(0, 2, 3, 1e-4, 5)["count"] == 0
