"""The headline render (512 x 512 pixels x 64 spp, at most 4 bounces, 78 -> 256 x 8 -> 2 network)
against the FP64 oracle, bounce by bounce, and renders spread over several waves.

ddf_render_trace records the query of every bounce of a 16 x 16-pixel block (16,384 paths) of the
full render. For each precision the test checks, against the oracle:
  * every bounce's query on the very ray the GPU queried: FP32 within 1e-5 (relative, floored at
    1), BF16 within 2e-2, FP8 against the model of its quantisation and with its FP64 error
    stated; hit decisions wherever the oracle's logit is clear of the precision's band;
  * every shading step: the next bounce's ray equals the oracle's hit point, offset and cosine
    sample (Sec. 3.1, Fig. 1) computed from the GPU's own query outputs, and the throughput;
  * every path's radiance: the value its recorded decisions imply, and (FP32) the radiance of the
    oracle's own FP64 path wherever none of its decisions lies within 1e-4 of the threshold; the
    pixels against the oracle image on pixels without such a path.
The multi-wave test renders more than 2^24 paths (two waves) and the same render in many small
waves: the images are identical bit for bit and the second wave's paths match the oracle."""

import numpy as np
import pytest
import torch

from ddf_synth import default_camera, init_weights
from oracle import mlp as omlp
from oracle.render import shade_step, trace_paths
from tests._helpers import BF16_ABS, LOGIT_MARGIN, NETS, ensure_built, fp32_close, net_weights

pytestmark = pytest.mark.gpu

HEAD = dict(F=12, W=256, L=8, seed=3, size=512, spp=64, bounces=4)   # the bench's render
BLOCK = (248, 248, 16)                                                # x0, y0, side of the traced block
FP8_ABS = 6e-2     # FP8 has no stated bound: distances against FP64 are held to 6e-2, decisions
                   # compared where |logit64| >= 6e-2 (measured errors: max ~0.03)


@pytest.fixture(scope="module")
def P():
    ensure_built()
    import paper_2306_16142_gb300 as P
    return P


def _block_pids(size, spp, x0, y0, side):
    ys, xs = np.meshgrid(np.arange(y0, y0 + side), np.arange(x0, x0 + side), indexing="ij")
    pix = (ys * size + xs).ravel()
    return pix, (pix[:, None] * spp + np.arange(spp)[None, :]).ravel()


def _normal_tolerance(Pm, o, w):
    """Per-row bound for the FP32 Eq. 3 normal: 1e-4 plus the rounding a float32 reverse pass can
    amplify when the gradient cancels, 1e-5 |g|_abs / |g|, where |g|_abs is the reverse pass of the
    same masks through |W| and |d features / d o| (the running-error bound of the sum) and g the
    FP64 gradient."""
    X, dX = omlp.encode(o, w, HEAD["F"])
    _, pres, acts = omlp.forward(Pm, X)
    gy = np.zeros((o.shape[0], 2))
    gy[:, 0] = 1.0
    _, gX = omlp.backward(Pm, pres, acts, gy)
    _, gXa = omlp.backward([(np.abs(Wl), bl) for Wl, bl in Pm], pres, acts, gy)
    g = np.zeros((o.shape[0], 3))
    ga = np.zeros((o.shape[0], 3))
    for f in range(X.shape[1]):
        if f % 6 < 3:
            g[:, f % 6] += gX[:, f] * dX[:, f]
            ga[:, f % 6] += np.abs(gXa[:, f] * dX[:, f])
    gn = np.linalg.norm(g, axis=1)
    return 1e-4 + 1e-5 * np.linalg.norm(ga, axis=1) / np.maximum(gn, 1e-300), gn


def _implied_radiance(tr, albedo, env):
    """Radiance each path's recorded decisions imply: k hits then a miss -> albedo^k env (in
    float32, as the kernel multiplies); a hit at the last bounce -> 0; no query -> env."""
    n, B, _ = tr.shape
    rad = np.full(n, np.float32(env), np.float32)
    done = np.zeros(n, bool)
    thr = np.ones(n, np.float32)
    for b in range(B):
        q = ~np.isnan(tr[:, b, 0]) & ~done
        hit = tr[:, b, 7] > 0
        m = q & ~hit
        rad[m] = thr[m] * np.float32(env)
        done |= m
        if b == B - 1:
            rad[q & hit] = 0.0
            done |= q & hit
        thr = np.where(q & hit, thr * np.float32(albedo), thr).astype(np.float32)
    return rad


def _check_shading(tr, pids, cam):
    """Bounce b + 1's ray is the oracle's move from bounce b's GPU outputs."""
    B = tr.shape[1]
    moved = 0
    for b in range(B - 1):
        cont = ~np.isnan(tr[:, b + 1, 0])
        if not cont.any():
            continue
        r0 = tr[cont, b].astype(np.float64)
        assert (r0[:, 7] > 0).all()                       # only paths that hit move on
        o2, w2 = shade_step(r0[:, 0:3], r0[:, 3:6], r0[:, 6], r0[:, 8:11], cam.seed, pids[cont], b + 1)
        r1 = tr[cont, b + 1].astype(np.float64)
        assert np.abs(r1[:, 0:3] - o2).max() <= 2e-6, np.abs(r1[:, 0:3] - o2).max()
        assert np.abs(r1[:, 3:6] - w2).max() <= 2e-5, np.abs(r1[:, 3:6] - w2).max()
        assert (tr[cont, b + 1, 11] == (tr[cont, b, 11] * np.float32(cam.albedo)).astype(np.float32)).all()
        # paths that hit and did not move on: only at the last bounce
        stopped = ~cont & ~np.isnan(tr[:, b, 0]) & (tr[:, b, 7] > 0)
        assert not stopped.any()
        moved += int(cont.sum())
    return moved


def _render_traced(P, precision):
    F, W, L, seed = HEAD["F"], HEAD["W"], HEAD["L"], HEAD["seed"]
    blob = init_weights(F, W, L, seed=seed)
    net = P.DDFNet(F, W, L, blob, precision)
    cam = default_camera(HEAD["size"], HEAD["size"], seed=1)
    pix, pids = _block_pids(HEAD["size"], HEAD["spp"], *BLOCK)
    img, tr, rad = net.render_trace(cam, HEAD["spp"], HEAD["bounces"], torch.from_numpy(pids).cuda())
    img_plain = net.render(cam, HEAD["spp"], HEAD["bounces"])
    net.device_status()
    assert torch.equal(img, img_plain)                   # tracing does not change the render
    return (blob, net, cam, pix, pids, img.cpu().numpy().ravel(), tr.cpu().numpy(), rad.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp8"])
def test_headline_render_bounce_by_bounce(P, precision):
    F, W, L = HEAD["F"], HEAD["W"], HEAD["L"]
    blob, net, cam, pix, pids, img, tr, rad = _render_traced(P, precision)
    Pm = omlp.unpack(blob, F, W, L)
    B = HEAD["bounces"]
    band = {"fp32": LOGIT_MARGIN, "bf16": BF16_ABS, "fp8": FP8_ABS}[precision]
    assert not np.isnan(tr[:, 0, 0]).any()               # the default camera: every ray enters the ball
    stats = []
    for b in range(B):
        q = ~np.isnan(tr[:, b, 0])
        if not q.any():
            continue
        r = tr[q, b]
        o, w = r[:, 0:3], r[:, 3:6]
        ref = omlp.query(Pm, o, w, F, with_normal=b < B - 1)
        clear = np.abs(ref["logit"]) >= band
        hit32 = r[:, 7] > 0
        mism = int((hit32[clear] != ref["hit"][clear]).sum())
        if precision == "fp32":
            assert fp32_close(r[:, 6], ref["dist"]).all(), np.abs(r[:, 6] - ref["dist"]).max()
            assert fp32_close(r[:, 7], ref["logit"]).all(), np.abs(r[:, 7] - ref["logit"]).max()
            assert mism == 0
            if b < B - 1 and hit32.any():
                tol, gn = _normal_tolerance(Pm, o[hit32], w[hit32])
                dn = np.abs(r[hit32, 8:11] - ref["normal"][hit32]).max(axis=1)
                ok = gn > 0
                assert (dn[ok] <= tol[ok]).all(), (dn[ok].max(), (dn[ok] > tol[ok]).sum())
                assert (dn[ok] <= 1e-4).mean() > 0.98
        elif precision == "bf16":
            assert np.abs(r[:, 6] - ref["dist"]).max() <= BF16_ABS
            assert np.abs(r[:, 7] - ref["logit"]).max() <= BF16_ABS
            assert mism == 0
        else:
            from tests._fp8_model import query_fp8
            m = query_fp8(Pm, o, w, F, net.fp8_scales())
            dm = np.abs(r[:, 6] - m["dist"])
            assert np.quantile(dm, 0.99) <= 5e-3 and dm.max() <= 3e-2, (np.quantile(dm, 0.99), dm.max())
            cm = np.abs(m["logit"]) >= 0.05
            assert (hit32[cm] == m["hit"][cm]).all()
            assert np.abs(r[:, 6] - ref["dist"]).max() <= FP8_ABS
            assert mism == 0
        if b < B - 1 and hit32.any():
            ang = np.degrees(np.arccos(np.clip(np.sum(r[hit32, 8:11] * ref["normal"][hit32], 1), -1, 1)))
            assert np.allclose(np.linalg.norm(r[hit32, 8:11], axis=1), 1, atol=1e-5)
            nstat = f", normal angle vs FP64 median {np.median(ang):.3f} p99 {np.percentile(ang, 99):.2f} deg"
        else:
            nstat = ""
        stats.append(f"bounce {b + 1}: {int(q.sum())} queries, max |d dist| "
                     f"{np.abs(r[:, 6] - ref['dist']).max():.2e}, {int((~clear).sum())} within the band{nstat}")
    moved = _check_shading(tr, pids, cam)
    assert moved > 500                                    # paths do bounce
    implied = _implied_radiance(tr, cam.albedo, cam.env)
    assert np.array_equal(rad, implied)
    # the pixels of the block are the means of their traced paths
    assert np.allclose(img[pix], rad.reshape(-1, HEAD["spp"]).mean(1), atol=1e-6)
    # the oracle's own FP64 paths
    own = trace_paths(lambda a, c: omlp.query(Pm, a, c, F), cam, HEAD["spp"], B, pids)
    if precision == "fp32":
        ok = own["min_abs_logit"] >= LOGIT_MARGIN
        assert ok.mean() > 0.95
        assert np.abs(rad[ok] - own["radiance"][ok]).max() <= 1e-6
        okp = ok.reshape(-1, HEAD["spp"]).all(1)
        ref_img = own["radiance"].reshape(-1, HEAD["spp"]).mean(1)
        assert np.abs(img[pix][okp] - ref_img[okp]).max() <= 1e-4
        print(f"FP32 headline block: exempt paths {1 - ok.mean():.4%}, exempt pixels {1 - okp.mean():.4%}")
    else:
        # first decisions are taken on the same camera rays (float32 vs float64 ray setup)
        first = np.abs(own["logit"]) >= band
        hit_first = tr[:, 0, 7] > 0
        assert (hit_first[first] == (own["logit"][first] > 0)).all()
        same = np.abs(rad - own["radiance"]) <= 1e-6
        print(f"{precision} headline block: {same.mean():.4f} of paths end with the FP64 path's radiance")
    print(f"{precision}: " + "; ".join(stats))


def test_render_over_several_waves(P):
    """1024 x 1024 pixels x 17 spp = 17,825,792 paths: two waves of at most 2^24 paths. The same
    render in waves of 2^20 and of 17,005 paths gives the same image bit for bit and the same
    per-bounce query counts; paths of the second wave (ids above 2^24) match the oracle."""
    name = "tiny_6x64x4"
    F, W, L, _, _ = NETS[name]
    blob = net_weights(name)
    net = P.DDFNet(F, W, L, blob)
    size, spp, B = 1024, 17, 3
    cam = default_camera(size, size, seed=4)
    a = net.render(cam, spp, B).cpu()
    sa = net.render_stats(B)
    assert sa[0] == size * size * spp and size * size * spp > (1 << 24)
    for wave in (1 << 20, 17 * 1000 + 5):
        net.set_wave(wave)
        b = net.render(cam, spp, B).cpu()
        assert torch.equal(a, b)
        assert net.render_stats(B) == sa
    net.set_wave(1 << 24)
    # pixels around the wave boundary (986,895 pixels per wave at 17 spp) and at the end
    first_wave_px = (1 << 24) // spp
    pix = np.concatenate([np.arange(first_wave_px - 40, first_wave_px + 40), np.arange(size * size - 60, size * size)])
    pids = (pix[:, None] * spp + np.arange(spp)[None, :]).ravel()
    img, tr, rad = net.render_trace(cam, spp, B, torch.from_numpy(pids).cuda())
    assert torch.equal(img.cpu(), a)
    img, tr, rad = img.cpu().numpy().ravel(), tr.cpu().numpy(), rad.cpu().numpy()
    Pm = omlp.unpack(blob, F, W, L)
    own = trace_paths(lambda o, w: omlp.query(Pm, o, w, F), cam, spp, B, pids)
    ok = own["min_abs_logit"] >= LOGIT_MARGIN
    assert ok.mean() > 0.9
    assert np.abs(rad[ok] - own["radiance"][ok]).max() <= 1e-6
    okp = ok.reshape(-1, spp).all(1)
    assert np.abs(img[pix][okp] - own["radiance"].reshape(-1, spp).mean(1)[okp]).max() <= 1e-4
    assert np.array_equal(rad, _implied_radiance(tr, cam.albedo, cam.env))
    _check_shading(tr, pids, cam)


def test_render_trace_arguments(P):
    F, W, L, _, _ = NETS["tiny_6x64x4"]
    net = P.DDFNet(F, W, L, net_weights("tiny_6x64x4"))
    with pytest.raises(P.DDFError):
        net.set_wave(0)
    with pytest.raises(P.DDFError):
        net.set_wave((1 << 24) + 1)
    cam = default_camera(8, 8)
    # ids outside the image stay NaN; an empty trace is a plain render
    img, tr, rad = net.render_trace(cam, 2, 2, torch.tensor([5, 10 ** 6], dtype=torch.int64, device="cuda"))
    assert np.isnan(tr[1].cpu().numpy()).all() and np.isnan(rad[1].item())
    assert not np.isnan(tr[0, 0, :8].cpu().numpy()).any()
    t0 = tr[0, 0].cpu().numpy()
    assert np.isnan(t0[8:11]).all() == (t0[7] <= 0)       # a normal exactly where the ray hit
    img2, _, _ = net.render_trace(cam, 2, 2, torch.empty(0, dtype=torch.int64, device="cuda"))
    assert torch.equal(img, img2)
