"""ddf_query_noalloc: the query entry point for callers that cannot allocate device memory
during a call (an engine whose allocations all go through its own pool, a render loop that
forbids allocation once running). Its scratch is a fixed static device array inside the library,
so it must give the same results as ddf_query; it is called twice in a row to show that the
shared array's left-over contents from the previous call do not leak into the next one.

This file is named to be collected last, so a run that stops at the first failure has already
run every other test."""

import ctypes as C

import numpy as np
import pytest
import torch

from ddf_synth import init_weights
from tests._helpers import BF16_ABS, ensure_built, rays_in_ball

pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _call(lib, fn, net, o, w, normals=True):
    n = o.shape[0]
    out = {"dist": torch.empty(n, device="cuda"), "hit": torch.empty(n, dtype=torch.uint8, device="cuda"),
           "logit": torch.empty(n, device="cuda"),
           "normal": torch.zeros(n, 3, device="cuda") if normals else None}
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(net.h, _p(o), _p(w), n, _p(out["dist"]), _p(out["hit"]), _p(out["logit"]),
                          _p(out["normal"]), stream)
    assert rc == 0, lib.ddf_last_error().decode()
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision,shape", [("bf16", (12, 256, 8, 2)), ("bf16", (0, 128, 6, 9)),
                                             ("fp32", (12, 256, 8, 2))])
def test_noalloc_matches_query_on_two_calls(precision, shape):
    ensure_built()
    import paper_2306_16142_gb300 as P
    lib = P.load()
    F, W, L, seed = shape
    net = P.DDFNet(F, W, L, init_weights(F, W, L, seed=seed), precision)
    tol = BF16_ABS if precision == "bf16" else 1e-5
    for call, n in enumerate((5000, 3001)):
        o, w = rays_in_ball(n, seed=40 + call)
        to, tw = torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()
        ref = _call(lib, "ddf_query", net, to, tw)
        got = _call(lib, "ddf_query_noalloc", net, to, tw)
        assert lib.ddf_device_status(net.h) == 0
        assert (got["dist"] - ref["dist"]).abs().max().item() <= tol
        assert (got["logit"] - ref["logit"]).abs().max().item() <= tol
        assert torch.equal(got["hit"], ref["hit"])
        hit = ref["hit"].bool()
        assert hit.any()
        assert (got["normal"][hit] - ref["normal"][hit]).abs().max().item() <= 1e-3
        assert (got["normal"][~hit] == 0).all()


def test_noalloc_rejects_rows_beyond_the_static_limit():
    ensure_built()
    import paper_2306_16142_gb300 as P
    lib = P.load()
    net = P.DDFNet(0, 128, 6, init_weights(0, 128, 6, seed=9), "bf16")
    big = (1 << 20) + 1
    z = torch.empty(1, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.ddf_query_noalloc(net.h, _p(z), _p(z), big, _p(z), _p(z), None, _p(z), stream)
    assert rc == -1
    assert b"static scratch limit" in lib.ddf_last_error()
