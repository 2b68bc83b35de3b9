"""GPU ray labelling against the FP64 brute-force oracle: hit, nearest-triangle index and
distance must be identical bit for bit, including stress rays through vertices and edges,
grazing rays and shared-edge ties, with the faces searched through the bounding-volume hierarchy
and by the sweep over all faces alike; and cases aimed at the hierarchy: duplicated faces (exact
ties in t, coincident centroids), a one-face mesh, axis-parallel rays and a 131,072-face mesh."""

import numpy as np
import pytest
import torch

from ddf_synth import icosphere, labelled_ray_set, torus_knot, uniform_sphere_rays
from oracle.label import label_rays
from tests._helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


@pytest.fixture(params=["bvh", "none"])
def accel(request):
    return request.param


def _gpu_label(P, V, F, o, w, accel="bvh"):
    mesh = P.DDFMesh(V, F, accel)
    out = mesh.label(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["stats"] = mesh.stats()
    return res


def _assert_exact(g, dist, hit, tri):
    assert (g["hit"] == hit).all(), np.nonzero(g["hit"] != hit)[0][:10]
    assert (g["tri"] == tri).all(), np.nonzero(g["tri"] != tri)[0][:10]
    assert (g["dist"].view(np.uint32) == dist.view(np.uint32)).all()


def _stress_rays(V, F, n, seed):
    """Rays from the bounding sphere aimed exactly at vertices, edge midpoints and edge
    points, plus grazing rays lying in a face's plane."""
    rng = np.random.default_rng(seed)
    Vd = V.astype(np.float64)
    k = rng.integers(0, F.shape[0], n)
    a = Vd[F[k, 0]]
    b = Vd[F[k, 1]]
    c = Vd[F[k, 2]]
    mode = rng.integers(0, 4, n)
    lam = rng.random(n)[:, None]
    tgt = np.where((mode == 0)[:, None], a,
          np.where((mode == 1)[:, None], 0.5 * (a + b),
          np.where((mode == 2)[:, None], lam * b + (1 - lam) * c, (a + b + c) / 3)))
    o = rng.normal(size=(n, 3))
    o /= np.linalg.norm(o, axis=1, keepdims=True)
    # grazing: origin in the face plane
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    graze = mode == 3
    inplane = o - np.sum(o * nrm, 1, keepdims=True) * nrm
    o[graze] = inplane[graze] / np.linalg.norm(inplane[graze], axis=1, keepdims=True)
    w = tgt - o
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    return o.astype(np.float32), w.astype(np.float32)


def test_label_icosphere_65536_bit_exact(P, accel):
    V, F = icosphere(2, 0.5)
    o, w = uniform_sphere_rays(65536, seed=11)
    g = _gpu_label(P, V, F, o, w, accel)
    d, h, t, _ = label_rays(V, F, o, w)
    _assert_exact(g, d, h, t)
    assert 0.03 < h.mean() < 0.2          # uniform rays from the unit sphere: ~6.7% meet r = 0.5


def test_label_stress_rays_bit_exact(P, accel):
    for V, F in (icosphere(2, 0.5), torus_knot(3, 2, 0.08, 64, 8)):
        o, w = _stress_rays(V, F, 8192, seed=3)
        g = _gpu_label(P, V, F, o, w, accel)
        d, h, t, _ = label_rays(V, F, o, w)
        _assert_exact(g, d, h, t)
        assert g["stats"]["retests"] > 0       # the edge / vertex rays need float64 re-tests


def test_label_shared_edge_ties(P, accel):
    V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], np.float32)
    F = np.array([[0, 2, 3], [0, 1, 2]], np.int32)
    xy = np.array([[0.5, 0.5], [0.25, 0.25], [0.0, 0.0], [1.0, 1.0], [0.75, 0.75], [0.3, 0.6]])
    o = np.concatenate([xy, np.ones((len(xy), 1))], 1).astype(np.float32)
    w = np.tile(np.array([[0, 0, -1]], np.float32), (len(xy), 1))
    g = _gpu_label(P, V, F, o, w, accel)
    d, h, t, _ = label_rays(V, F, o, w)
    _assert_exact(g, d, h, t)
    assert (t[:5] == 0).all()


def test_label_ragged_and_tiny(P, accel):
    V, F = torus_knot(3, 2, 0.08, 32, 4)     # 256 triangles: exactly one tile
    for n in (1, 31, 513, 1000):
        o, w = uniform_sphere_rays(n, seed=n)
        g = _gpu_label(P, V, F, o, w, accel)
        _assert_exact(g, *label_rays(V, F, o, w)[:3])
    V2, F2 = V, F[:257]                        # ragged triangle tile
    o, w = uniform_sphere_rays(777, seed=5)
    g = _gpu_label(P, V2, F2, o, w, accel)
    _assert_exact(g, *label_rays(V2, F2, o, w)[:3])


def test_label_knot_training_mix_bit_exact(P, accel):
    V, F = torus_knot(3, 2, 0.08, 256, 16)     # 8,192 triangles
    o, w = labelled_ray_set(V, F, 16384, seed=11)
    g = _gpu_label(P, V, F, o, w, accel)
    d, h, t, _ = label_rays(V, F, o, w)
    _assert_exact(g, d, h, t)


def test_label_full_size_sampled(P, accel):
    """2^20 training rays against the 8,192-triangle knot in one launch; 512 sampled rows."""
    V, F = torus_knot(3, 2, 0.08, 256, 16)
    o, w = labelled_ray_set(V, F, 1 << 20, seed=11)
    g = _gpu_label(P, V, F, o, w, accel)
    idx = np.random.default_rng(1).choice(o.shape[0], 512, replace=False)
    d, h, t, _ = label_rays(V, F, o[idx], w[idx])
    _assert_exact({k: v[idx] for k, v in g.items() if k != "stats"}, d, h, t)
    # re-tests are rare: well under 1% of rays
    assert g["stats"]["retests"] < 0.01 * o.shape[0] * 10


def test_bvh_duplicated_faces_tie_to_the_lower_index(P):
    """Every face twice (the copy 1,280 indices later): every hit is an exact tie in t and must go
    to the original; the copies' centroids coincide, which the hierarchy splits arbitrarily."""
    V, F = icosphere(3, 0.5)
    F2 = np.concatenate([F, F[::-1]]).astype(np.int32)
    o, w = _stress_rays(V, F, 8192, seed=9)
    for accel in ("bvh", "none"):
        g = _gpu_label(P, V, F2, o, w, accel)
        d, h, t, _ = label_rays(V, F2, o, w)
        _assert_exact(g, d, h, t)
    assert h.mean() > 0.5


def test_bvh_single_face_and_axis_parallel_rays(P):
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    F = np.array([[0, 1, 2]], np.int32)
    rng = np.random.default_rng(2)
    xy = rng.uniform(-0.2, 1.2, (4096, 2))
    o = np.concatenate([xy, np.full((4096, 1), 2.0)], 1).astype(np.float32)
    w = np.tile(np.array([[0, 0, -1]], np.float32), (4096, 1))       # two zero components
    g = _gpu_label(P, V, F, o, w, "bvh")
    _assert_exact(g, *label_rays(V, F, o, w)[:3])
    # rays in the face's plane and along the box faces
    o2 = np.concatenate([xy, np.zeros((4096, 1))], 1).astype(np.float32)
    w2 = np.tile(np.array([[1, 0, 0]], np.float32), (4096, 1))
    g2 = _gpu_label(P, V, F, o2, w2, "bvh")
    _assert_exact(g2, *label_rays(V, F, o2, w2)[:3])


def test_bvh_matches_the_sweep_on_a_large_mesh(P):
    """2^18 training rays against the 131,072-face knot: the hierarchy's labels equal the sweep's."""
    V, F = torus_knot(3, 2, 0.08, 1024, 64)
    o, w = labelled_ray_set(V, F, 1 << 18, seed=4)
    a = _gpu_label(P, V, F, o, w, "bvh")
    b = _gpu_label(P, V, F, o, w, "none")
    for k in ("hit", "tri"):
        assert np.array_equal(a[k], b[k])
    assert (a["dist"].view(np.uint32) == b["dist"].view(np.uint32)).all()
    idx = np.random.default_rng(3).choice(o.shape[0], 256, replace=False)
    d, h, t, _ = label_rays(V, F, o[idx], w[idx])
    _assert_exact({k: v[idx] for k, v in a.items() if k != "stats"}, d, h, t)
