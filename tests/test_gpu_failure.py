"""Failure detection without a GPU fault: a bounded device wait that nothing satisfies gives
up, raises the device flag and returns; the host reads DDF_ERR_TIMEOUT and the context keeps
working. Host-side failures (bad arguments, missing library) are covered in test_abi.py."""

import numpy as np
import pytest
import torch

from ddf_synth import init_weights
from oracle import mlp as omlp
from tests._helpers import BF16_ABS, ensure_built, rays_in_ball

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    ensure_built()
    import paper_2306_16142_gb300 as P
    from paper_2306_16142_gb300 import _abi
    lib = P.load()
    assert lib.ddf_selftest_wait(20, 1) == _abi.DDF_OK                 # signal arrives: completes
    assert lib.ddf_selftest_wait(20, 0) == _abi.DDF_ERR_TIMEOUT        # lost signal: gives up
    assert b"gave up" in lib.ddf_last_error()
    # the context still runs the tensor-core path correctly afterwards
    F, W, L = 12, 256, 4
    blob = init_weights(F, W, L, seed=1)
    net = P.DDFNet(F, W, L, blob, "bf16")
    o, w = rays_in_ball(1000, seed=2)
    out = net.query(torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda())
    net.device_status()
    ref = omlp.query(omlp.unpack(blob, F, W, L), o, w, F, with_normal=False)
    assert np.abs(out["dist"].cpu().numpy() - ref["dist"]).max() <= BF16_ABS
