"""GPU grouped multi-object query: every object's rows equal the single-object BF16 query on
the same rays (same arithmetic, one launch per width class: 128, 256 and 512), within the BF16
tolerance of the FP64 oracle; ragged and empty objects; CUDA-graph capture and replay after the
device-side offsets change; the launch-shape autotuner (ring depth and grid) and its cache."""

import numpy as np
import pytest
import torch

from ddf_synth import init_weights
from oracle import mlp as omlp
from tests._helpers import BF16_ABS, ensure_built, rays_in_ball

pytestmark = pytest.mark.gpu

# (in_freqs, width, hidden_layers, seed)
OBJS = [(12, 256, 8, 100), (12, 128, 4, 101), (12, 256, 5, 102), (12, 128, 8, 103), (12, 256, 6, 104),
        (0, 128, 6, 105), (12, 512, 4, 106), (16, 512, 8, 107), (12, 512, 6, 108)]


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


def _setup(P, counts, seed=0):
    nets = [P.DDFNet(F, W, L, init_weights(F, W, L, seed=s), "bf16") for F, W, L, s in OBJS]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    o, w = rays_in_ball(int(off[-1]), seed=seed)
    return nets, off, o, w


def test_grouped_equals_single_object_queries(P):
    counts = [1000, 1, 0, 5000, 129, 3000, 4000, 127, 1]
    nets, off, o, w = _setup(P, counts)
    grp = P.DDFGroup(nets)
    to, tw = torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()
    toff = torch.from_numpy(off).cuda()
    out = grp.query(toff, to, tw)
    grp.status()
    for i, (F, W, L, s) in enumerate(OBJS):
        a, b = int(off[i]), int(off[i + 1])
        if a == b:
            continue
        ref = nets[i].query(to[a:b].contiguous(), tw[a:b].contiguous())
        assert torch.equal(out["dist"][a:b], ref["dist"])
        assert torch.equal(out["logit"][a:b], ref["logit"])
        assert torch.equal(out["hit"][a:b], ref["hit"])
        r = omlp.query(omlp.unpack(init_weights(F, W, L, seed=s), F, W, L), o[a:b], w[a:b], F, with_normal=False)
        assert np.abs(out["dist"][a:b].cpu().numpy() - r["dist"]).max() <= BF16_ABS


def test_grouped_graph_replay_follows_device_offsets(P):
    counts = [2000, 700, 100, 4000, 1, 900, 300, 2000, 0]
    nets, off, o, w = _setup(P, counts, seed=3)
    grp = P.DDFGroup(nets)
    to, tw = torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()
    toff = torch.from_numpy(off).cuda()
    out = grp._out(o.shape[0], "cuda")
    grp.capture(toff, to, tw, out)
    grp.replay()
    torch.cuda.synchronize()
    ref = grp.query(toff, to, tw)
    torch.cuda.synchronize()
    assert torch.equal(out["dist"], ref["dist"]) and torch.equal(out["hit"], ref["hit"])
    # new ray counts written on the device; the same graph serves them
    counts2 = [10, 4000, 0, 1200, 2400, 1, 0, 1, 2300]
    off2 = np.concatenate([[0], np.cumsum(counts2)]).astype(np.int64)
    assert off2[-1] <= o.shape[0]
    toff.copy_(torch.from_numpy(off2).cuda())
    out["dist"].fill_(float("nan"))
    grp.replay()
    torch.cuda.synchronize()
    ref2 = grp.query(toff, to, tw)
    torch.cuda.synchronize()
    n2 = int(off2[-1])
    assert torch.equal(out["dist"][:n2], ref2["dist"][:n2])
    grp.status()


def test_autotuner_and_cache(P, tmp_path):
    counts = [3000] * len(OBJS)
    nets, off, o, w = _setup(P, counts, seed=5)
    grp = P.DDFGroup(nets)
    to, tw = torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()
    toff = torch.from_numpy(off).cuda()
    out = grp._out(o.shape[0], "cuda")
    cache = str(tmp_path / "tune.txt")
    cfg = grp.autotune(toff, to, tw, out, reps=2, cache_path=cache)
    assert [c[0] for c in cfg] == [128, 256, 512]
    assert all(c[1] >= 2 and c[2] > 0 for c in cfg)
    assert cfg[2][1] in (2, 3)
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 3
    grp2 = P.DDFGroup(nets)
    assert grp2.autotune(toff, to, tw, out, reps=2, cache_path=cache) == cfg   # read back, no new lines
    assert len(open(cache).read().strip().splitlines()) == 3
    res = grp2.query(toff, to, tw)
    ref = grp.query(toff, to, tw)
    torch.cuda.synchronize()
    assert torch.equal(res["dist"], ref["dist"])
