"""ddf_query_noalloc: the query entry point for callers that cannot allocate device memory
during a call (an engine whose allocations all go through its own pool, a render loop that
forbids allocation once running). Its scratch is a fixed static device array inside the library.

Each case builds a fresh handle and calls ddf_query_noalloc before anything else touches it, twice
in a row (so the shared array's left-over contents from the first call meet the second), and only
then calls ddf_query for the comparison. That the entry point allocates nothing is shown on the
device itself: the free device memory (cudaMemGetInfo) is the same before and after a batch of
2^20-row calls, while one ddf_query of the same size on the same handle, which grows the handle's
4 MiB hit-row list, visibly lowers it.

This file is named to be collected last, so a run that stops at the first failure has already
run every other test."""

import ctypes as C

import numpy as np
import pytest
import torch

from ddf_synth import init_weights
from tests._helpers import BF16_ABS, ensure_built, rays_in_ball

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16": BF16_ABS, "fp8": BF16_ABS}


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _lib():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P, P.load()


def _out(n, normals=True):
    return {"dist": torch.empty(n, device="cuda"), "hit": torch.empty(n, dtype=torch.uint8, device="cuda"),
            "logit": torch.empty(n, device="cuda"),
            "normal": torch.zeros(n, 3, device="cuda") if normals else None}


def _call(lib, fn, net, o, w, out):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(net.h, _p(o), _p(w), o.shape[0], _p(out["dist"]), _p(out["hit"]), _p(out["logit"]),
                          _p(out["normal"]), stream)
    assert rc == 0, lib.ddf_last_error().decode()
    return out


def _rays(n, seed):
    o, w = rays_in_ball(n, seed=seed)
    return torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()


def _weights_with_hits(F, W, L, seed):
    """Seeded weights whose hit-logit bias is moved so that about a third of the rays in the
    ball hit (a random network of width 512 hardly ever does), from the FP64 oracle's logits."""
    from oracle import mlp as omlp
    blob = init_weights(F, W, L, seed=seed)
    o, w = rays_in_ball(4096, seed=7)
    lg = omlp.query(omlp.unpack(blob, F, W, L), o, w, F, with_normal=False)["logit"]
    blob[-1] -= np.float32(np.quantile(lg, 0.67))
    return blob


@pytest.mark.parametrize("precision,shape", [("bf16", (12, 256, 8, 2)), ("bf16", (0, 128, 6, 9)),
                                             ("bf16", (16, 512, 4, 5)), ("fp8", (12, 256, 8, 2)),
                                             ("fp8", (0, 128, 6, 9)), ("fp32", (12, 256, 8, 2))])
def test_noalloc_matches_query_on_two_calls(precision, shape):
    P, lib = _lib()
    F, W, L, seed = shape
    net = P.DDFNet(F, W, L, _weights_with_hits(F, W, L, seed), precision)
    calls = [(5000, 40), (3001, 41)]
    rays = [_rays(n, s) for n, s in calls]
    got = [_call(lib, "ddf_query_noalloc", net, o, w, _out(o.shape[0])) for o, w in rays]   # first, fresh handle
    torch.cuda.synchronize()
    assert lib.ddf_device_status(net.h) == 0
    tol = TOL[precision]
    for (o, w), g in zip(rays, got):
        ref = _call(lib, "ddf_query", net, o, w, _out(o.shape[0]))
        torch.cuda.synchronize()
        assert (g["dist"] - ref["dist"]).abs().max().item() <= tol
        assert (g["logit"] - ref["logit"]).abs().max().item() <= tol
        assert torch.equal(g["hit"], ref["hit"])
        hit = ref["hit"].bool()
        assert hit.any()
        assert (g["normal"][hit] - ref["normal"][hit]).abs().max().item() <= 1e-3
        assert (g["normal"][~hit] == 0).all()


@pytest.mark.parametrize("precision,shape", [("bf16", (12, 256, 8, 2)), ("fp8", (12, 256, 8, 2)),
                                             ("bf16", (16, 512, 4, 5))])
def test_noalloc_allocates_nothing(precision, shape):
    P, lib = _lib()
    F, W, L, seed = shape
    net = P.DDFNet(F, W, L, _weights_with_hits(F, W, L, seed), precision)
    n = 1 << 20
    o, w = _rays(n, 42)
    out, out2 = _out(n), _out(n)
    _call(lib, "ddf_query_noalloc", net, o, w, out)     # the first call looks the array up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(8):
        _call(lib, "ddf_query_noalloc", net, o, w, out)
    torch.cuda.synchronize()
    assert lib.ddf_device_status(net.h) == 0
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert out["hit"].sum().item() > 0
    # control: ddf_query grows the handle's hit-row list (4 MiB for 2^20 rows), which shows up
    _call(lib, "ddf_query", net, o, w, out2)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free0 - free2 >= 4 << 20, (free0, free2)


def test_noalloc_row_limit_applies_only_where_the_array_is_used():
    P, lib = _lib()
    net = P.DDFNet(0, 128, 6, init_weights(0, 128, 6, seed=9), "bf16")
    big = (1 << 20) + 1
    z = torch.empty(1, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.ddf_query_noalloc(net.h, _p(z), _p(z), big, _p(z), _p(z), None, _p(z), stream)
    assert rc == -1
    assert b"static scratch limit" in lib.ddf_last_error()
    # without normals the query needs no scratch: any n, and the same results as ddf_query
    o, w = _rays(big, 43)
    a = _call(lib, "ddf_query_noalloc", net, o, w, _out(big, normals=False))
    b = _call(lib, "ddf_query", net, o, w, _out(big, normals=False))
    torch.cuda.synchronize()
    assert torch.equal(a["dist"], b["dist"]) and torch.equal(a["hit"], b["hit"])
