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


@pytest.mark.parametrize("accel", ["bvh", "none"])
@pytest.mark.parametrize("name", list(CASES))
def test_sampler_matches_oracle_bit_for_bit(P, name, accel):
    make, (s_fc, s_dr, s_p, eps, seed) = CASES[name]
    V, T = make()
    mesh = P.DDFMesh(V, T, accel)
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


def _box(a):
    a = np.float32(a)
    V = np.array([[x, y, z] for x in (-a, a) for y in (-a, a) for z in (-a, a)], np.float32)
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    F = []
    for q in quads:
        F += [[q[0], q[1], q[2]], [q[0], q[2], q[3]]]
    return V, np.array(F, np.int32)


POV_CASES = {
    # the paper's 10 x 5 cameras; an odd film (a centre pixel); a wide field of view whose corner
    # rays miss the unit ball (origin left at the eye); a camera inside the ball
    "icosphere": (lambda: icosphere(2, 0.5), dict(n_az=10, n_pol=5, res=12)),
    "knot": (lambda: torus_knot(3, 2, 0.08, 64, 8), dict(n_az=10, n_pol=5, res=9)),
    "box_wide": (lambda: _box(0.4), dict(n_az=7, n_pol=3, res=16, dist=2.5, tan_half_fov=1.2)),
    "inside": (lambda: _box(0.3), dict(n_az=3, n_pol=2, res=8, dist=0.8, tan_half_fov=0.5)),
}


@pytest.mark.parametrize("name", list(POV_CASES))
def test_pov_matches_oracle_bit_for_bit(P, name):
    make, kw = POV_CASES[name]
    V, T = make()
    g = P.DDFMesh(V, T).sample_pov(**kw)
    torch.cuda.synchronize()
    r = S.sample_pov(V, T, **kw)
    n = kw["n_az"] * kw["n_pol"] * kw["res"] ** 2
    assert g["o"].shape[0] == n == r["o"].shape[0]
    assert np.array_equal(g["w"].cpu().numpy(), r["w"])
    assert np.array_equal(g["o"].cpu().numpy(), r["o"])
    assert np.array_equal(g["hit"].cpu().numpy(), r["hit"])
    assert np.array_equal(g["dist"].cpu().numpy(), r["dist"])
    print(f"{name}: {n} rays, {int(r['hit'].sum())} hits")
    if name == "box_wide":
        assert (np.linalg.norm(r["o"].astype(np.float64), axis=1) > 2.0).any()   # rays that miss the ball


def test_pov_rejects_bad_arguments(P):
    V, T = _box(0.4)
    mesh = P.DDFMesh(V, T)
    for kw in (dict(dist=0.0), dict(dist=float("inf")), dict(tan_half_fov=0.0), dict(tan_half_fov=float("nan")),
               dict(res=-1)):
        with pytest.raises(P.DDFError):
            mesh.sample_pov(**kw)
    assert mesh.sample_pov(n_az=0)["o"].shape[0] == 0


@pytest.mark.parametrize("name,n,seed", [("icosphere", 20000, 3), ("knot", 5000, 8), ("box", 7777, 1)])
def test_random_matches_oracle_bit_for_bit(P, name, n, seed):
    V, T = {"icosphere": lambda: icosphere(2, 0.5), "knot": lambda: torus_knot(3, 2, 0.08, 64, 8),
            "box": lambda: _box(0.4)}[name]()
    g = P.DDFMesh(V, T).sample_random(n, seed)
    torch.cuda.synchronize()
    r = S.sample_random(V, T, n, seed)
    for k in ("o", "w", "dist", "hit"):
        assert np.array_equal(g[k].cpu().numpy(), r[k]), k
    assert 0.05 < r["hit"].mean() < 0.95
