"""The query with normals through ddf_query and through ddf_query_noalloc: BF16 at widths 128 / 256
(the same forward and normal launches, the hit-row list in the library's static array instead of
the handle's) and FP32 (ddf_query lists the hit rows and runs the reverse pass on them alone, the
allocation-free form runs it inside the forward launch on every tile that holds a hit). The
outputs, normals included, are equal bit for bit, on two calls in a row and on ragged tiles of
hit rows."""

import ctypes as C

import numpy as np
import pytest
import torch

from ddf_synth import init_weights
from tests._helpers import ensure_built, rays_in_ball

pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _call(lib, fn, net, o, w):
    n = o.shape[0]
    out = {"dist": torch.empty(n, device="cuda"), "hit": torch.empty(n, dtype=torch.uint8, device="cuda"),
           "logit": torch.empty(n, device="cuda"), "normal": torch.full((n, 3), 7.0, device="cuda")}
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(net.h, _p(o), _p(w), n, _p(out["dist"]), _p(out["hit"]), _p(out["logit"]),
                          _p(out["normal"]), stream)
    assert rc == 0, lib.ddf_last_error().decode()
    return out


@pytest.mark.parametrize("precision,shape", [("bf16", (12, 256, 8, 2)), ("bf16", (0, 128, 6, 9)),
                                             ("bf16", (16, 256, 3, 4)), ("fp32", (12, 256, 8, 2)),
                                             ("fp32", (0, 128, 6, 9))])
@pytest.mark.parametrize("n", [5000, 70001])
def test_query_and_noalloc_agree_bit_for_bit(precision, shape, n):
    ensure_built()
    import paper_2306_16142_gb300 as P
    lib = P.load()
    F, W, L, seed = shape
    blob = init_weights(F, W, L, seed=seed)
    # the hit-logit bias moved so that about 40% of the rays hit (ragged hit tiles), from the FP64
    # oracle's logits of a sample of the same rays
    from oracle import mlp as omlp
    os_, ws_ = rays_in_ball(4096, seed=seed + 100)
    lg = omlp.query(omlp.unpack(blob, F, W, L), os_, ws_, F, with_normal=False)["logit"]
    blob[-1] -= np.float32(np.quantile(lg, 0.6))
    net = P.DDFNet(F, W, L, blob, precision)
    o, w = [torch.from_numpy(x).cuda() for x in rays_in_ball(n, seed=seed + 100)]
    first = _call(lib, "ddf_query", net, o, w)
    again = _call(lib, "ddf_query", net, o, w)            # the second call reuses the buffers
    static = _call(lib, "ddf_query_noalloc", net, o, w)
    torch.cuda.synchronize()
    assert lib.ddf_device_status(net.h) == 0
    hit = static["hit"].bool()
    frac = hit.float().mean().item()
    print(f"W={W} L={L} n={n}: hit fraction {frac:.3f}")
    assert 0.02 < frac < 0.98
    for out in (first, again):
        assert torch.equal(out["hit"], static["hit"])
        assert torch.equal(out["dist"], static["dist"])
        assert torch.equal(out["normal"][hit], static["normal"][hit])
