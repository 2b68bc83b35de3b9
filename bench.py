"""Benchmark of the DDF hot path on GB300.

One step = one full render of the single-object workload (the modified path tracer of the
paper's Sec. 1 / Fig. 1): 512 x 512 pixels x 64 samples, at most 4 bounces, a 78 -> 256 x 8 -> 2
network (12-frequency encoding, seeded weights: the workload the parity tests check path by path),
one wave of 2^24 paths: camera rays, one batched field query per bounce (distance, hit, Eq. 3
normal), shading + compaction, per-pixel accumulation - every step in libddf.so's kernels. The
same render of the network the run trains first (Sec. 5.1 / 5.2 in this build's reading: 6,000
BF16 tensor-core Adam steps of batch 65,536 on 2^20 rays labelled by ddf_label_rays against the
8,192-face (3,2) torus knot) is reported beside it.

Prints ONE JSON line (rank 0): samples/s over the timed steps (device time, CUDA events, max over
ranks), the dominant kernel's roofline, the end-to-end figure through the public API with the
image read back to pinned host memory, the FP64 oracle timed on the host cores on a bounded
sample, SM clocks sampled during the timed region, the FP32 / BF16 / FP8 query errors against the
oracle on 2^20 of the render's own query rays, and the other hot-path rows, the full large render
(1920 x 1080 x 256 spp, <= 8 bounces, 102 -> 512 x 8 -> 2; FP32 / BF16 / FP8) among them.

--impl reference times the FP64 oracle itself on the host (a bounded sample per step).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DDF ray queries/s and render samples/s, BF16/FP8 vs FP32 on 1 GB300 at stated error"
WORKLOAD = dict(width=512, height=512, spp=64, bounces=4, in_freqs=12, hidden=256, layers=8, seed=3)


TRAIN = dict(rays=1 << 20, batch=65536, steps=6000, lr=3e-3, seed_init=2, seed_rays=11)
LARGE = dict(width=1920, height=1080, spp=256, bounces=8, in_freqs=16, hidden=512, layers=8, seed=5)


def workload_name(w, trained=False):
    E = 6 + 6 * w["in_freqs"]
    net = ("trained on 2^20 labelled rays of the 8,192-face (3,2) torus knot" if trained else "seeded weights")
    return (f"single-object render {w['width']}x{w['height']} x {w['spp']} spp, <= {w['bounces']} bounces, "
            f"{E}->{w['hidden']}x{w['layers']}->2 DDF MLP ({net})")


def fwd_flops(E, W, L):
    return 2.0 * (E * W + (L - 1) * W * W + 2 * W)


def bwd_flops(E, W, L):
    # reverse pass to the input for a hit row: W x W per hidden layer after the first, W x E last
    return 2.0 * ((L - 1) * W * W + W * E)


# ncu-measured DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per row of the BF16
# query kernels, captured on one bounce-1 launch each of the 512 x 512 x 32 spp render (whose rays
# exceed the L2): mlp_pair_kernel<256> forward over 8,388,608 rows, mlp_pairn_kernel<256> normals
# over 1,265,231 hit rows (profiles/bf16_query_render512x512.md). A render's traffic is these
# times its rows; to be measured again whenever those kernels change.
QUERY_DRAM_BYTES_PER_FWD_ROW = (203441920 + 51336960) / 8388608
QUERY_DRAM_BYTES_PER_NRM_ROW = (40118784 + 855296) / 1265231


def query_traffic_per_bounce(stats, bounces):
    """DRAM bytes of the BF16 query launches per bounce query: forward rows are every bounce's live
    rays, normal rows the hits, i.e. the next bounce's rays."""
    render_bytes = QUERY_DRAM_BYTES_PER_FWD_ROW * sum(stats) + QUERY_DRAM_BYTES_PER_NRM_ROW * sum(stats[1:])
    return render_bytes / bounces


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(torch, ms, world, device="cuda"):
    """The slowest rank's time: every rank's timed region is bracketed by barriers, so the job takes
    as long as its slowest rank (an all-reduce MAX over the process group when world > 1)."""
    if world > 1:
        t = torch.tensor([float(ms)], device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = t.item()
    return ms


def whole_job_rate(units_per_rank_step, world, steps, ms):
    """Units per second of the whole job: every rank processes units_per_rank_step units per step
    (weak scaling), in ms milliseconds for `steps` steps (the slowest rank's time)."""
    return units_per_rank_step * world * steps / (ms / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_render_sample(w, blob, n_paths, precision_note=""):
    """Time the FP64 oracle on n_paths paths of the same render (bounded CPU work)."""
    import numpy as np
    from ddf_synth import default_camera
    from oracle import mlp as omlp
    from oracle.render import trace_paths
    cam = default_camera(w["width"], w["height"], seed=1)
    P = omlp.unpack(blob, w["in_freqs"], w["hidden"], w["layers"])
    total = w["width"] * w["height"] * w["spp"]
    pids = np.random.default_rng(0).choice(total, n_paths, replace=False)
    nq = [0]

    def q(o, d):
        nq[0] += o.shape[0]
        return omlp.query(P, o, d, w["in_freqs"])

    t0 = time.perf_counter()
    trace_paths(q, cam, w["spp"], w["bounces"], pids)
    dt = time.perf_counter() - t0
    return dt, nq[0]


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from ddf_synth import init_weights
    w = WORKLOAD
    blob = init_weights(w["in_freqs"], w["hidden"], w["layers"], seed=w["seed"])
    n_paths = args.ref_paths
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_render_sample(w, blob, max(64, n_paths // 16))
    times, nqs = [], []
    for _ in range(args.steps):
        dt, nq = oracle_render_sample(w, blob, n_paths)
        times.append(dt)
        nqs.append(nq)
    tot = sum(times)
    value = n_paths * args.steps / tot
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(w, trained=False), "parallelism": "host cores (numpy FP64 oracle)"},
            "queries_per_s": sum(nqs) / tot,
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{n_paths} random paths of the {w['width']}x{w['height']}x{w['spp']} "
                                       f"render per step"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def train_knot_field(P, torch, np):
    """The config-2 network trained by the library: 2^20 rays (half uniform on the bounding sphere,
    half aimed at the knot's surface with 0.05 rad of jitter) labelled by ddf_label_rays against the
    8,192-face (3,2) torus knot, TRAIN["steps"] BF16 tensor-core Adam steps of batch 65,536 over
    reshuffled epochs, learning rate TRAIN["lr"] with a cosine decay. Returns the FP32 master
    weights (host blob) and the training record (loss curve, held-out hit accuracy and L1)."""
    from ddf_synth import init_weights, labelled_ray_set, torus_knot
    V, F = torus_knot(3, 2, 0.08, 256, 16)
    mesh = P.DDFMesh(V, F)
    o, w = labelled_ray_set(V, F, TRAIN["rays"], seed=TRAIN["seed_rays"])
    to, tw = torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()
    lab = mesh.label(to, tw)
    dgt, hgt = lab["dist"], lab["hit"]
    net = P.DDFNet(12, 256, 8, init_weights(12, 256, 8, seed=TRAIN["seed_init"]), "bf16")
    g = torch.Generator(device="cuda").manual_seed(0)
    loss = torch.empty((), device="cuda")
    B, nb = TRAIN["batch"], TRAIN["rays"] // TRAIN["batch"]
    steps, curve = TRAIN["steps"], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    perm = None
    for st in range(steps):
        if st % nb == 0:
            perm = torch.randperm(TRAIN["rays"], device="cuda", generator=g)
        idx = perm[(st % nb) * B:(st % nb + 1) * B]
        lr = max(TRAIN["lr"] * 0.5 * (1.0 + math.cos(math.pi * st / steps)), TRAIN["lr"] * 0.01)
        net.train_step(to[idx], tw[idx], dgt[idx], hgt[idx], lr=lr, loss=loss)
        if st % 500 == 0 or st == steps - 1:
            curve.append((st, round(float(loss.item()), 5)))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    net.device_status()
    ho, hw = labelled_ray_set(V, F, 1 << 16, seed=TRAIN["seed_rays"] + 1)
    tho, thw = torch.from_numpy(ho).cuda(), torch.from_numpy(hw).cuda()
    hl = mesh.label(tho, thw)
    out = net.query(tho, thw)
    hit, ht = out["hit"].bool(), hl["hit"].bool()
    both = hit & ht
    info = {"workload": "78 -> 256 x 8 -> 2 from Xavier seed 2, 2^20 rays labelled against the 8,192-face (3,2) "
                        "knot, batch 65,536, Adam (cosine learning rate from 3e-3), BF16 tensor-core steps",
            "steps": steps, "s": dt, "ms_per_step": dt * 1e3 / steps, "loss_curve": curve,
            "heldout_hit_accuracy": float((hit == ht).float().mean().item()),
            "heldout_l1_on_hits": float((out["dist"][both] - hl["dist"][both]).abs().mean().item()),
            "labelled_hit_fraction": float(hgt.float().mean().item())}
    return net.get_weights().cpu().numpy(), info


def render_query_rays(P, torch, np, net, cam, spp, bounces, n_rays, seed):
    """n_rays of the rays a render actually queries: ddf_render_trace of n_rays random paths, every
    recorded bounce's (o, w), then n_rays of those drawn uniformly (so each bounce is represented in
    proportion to its share of the render's queries). Returns (o, w, rays per bounce)."""
    total = cam.width * cam.height * spp
    rng = np.random.default_rng(seed)
    pids = np.sort(rng.choice(total, n_rays, replace=False)).astype(np.int64)
    _, tr, _ = net.render_trace(cam, spp, bounces, torch.from_numpy(pids).cuda())
    tr = tr[:, :, 0:6].cpu().numpy()
    q = ~np.isnan(tr[:, :, 0])
    rays = tr[q]
    bounce = np.nonzero(q)[1]
    pick = np.sort(rng.choice(rays.shape[0], min(n_rays, rays.shape[0]), replace=False))
    o = np.ascontiguousarray(rays[pick, 0:3])
    w = np.ascontiguousarray(rays[pick, 3:6])
    return o, w, np.bincount(bounce[pick], minlength=bounces).tolist()


def oracle_query_job(blob, F, W, L, o, w, hit_any, chunk=1 << 15):
    """FP64 oracle outputs on the given rays (runs in a spawned worker): distance and logit of
    every row, the Eq. 3 normal of the rows in hit_any."""
    import numpy as np
    from oracle import mlp as omlp
    Pm = omlp.unpack(blob, F, W, L)
    n = o.shape[0]
    dist, logit = np.empty(n), np.empty(n)
    for a in range(0, n, chunk):
        r = omlp.query(Pm, o[a:a + chunk], w[a:a + chunk], F, with_normal=False)
        dist[a:a + chunk], logit[a:a + chunk] = r["dist"], r["logit"]
    rows = np.nonzero(hit_any)[0]
    normal = np.zeros((rows.size, 3))
    for a in range(0, rows.size, chunk):
        rr = rows[a:a + chunk]
        normal[a:a + chunk] = omlp.query(Pm, o[rr], w[rr], F)["normal"]
    return dist, logit, rows, normal


def error_stats(gpu, ref, band, bound):
    """Errors of one precision's query outputs against the oracle's on the same rays; bound is the
    precision's distance tolerance (FP32: relative, floored at 1; BF16: absolute; FP8: stated)."""
    import numpy as np
    dist64, logit64, rows, normal64 = ref
    dd = np.abs(gpu["dist"].astype(np.float64) - dist64)
    dl = np.abs(gpu["logit"].astype(np.float64) - logit64)
    rel = dd / np.maximum(np.abs(dist64), 1.0)
    h64 = logit64 > 0
    hit = gpu["hit"].astype(bool)
    clear = np.abs(logit64) >= 1e-4
    off = np.abs(logit64) >= band
    both = hit[rows] & (logit64[rows] > 0)
    cos = np.clip(np.sum(gpu["normal"][rows][both].astype(np.float64) * normal64[both], 1), -1, 1)
    ang = np.degrees(np.arccos(cos)) if both.any() else np.zeros(1)
    return {"max_abs_dist": float(dd.max()), "p99_abs_dist": float(np.percentile(dd, 99)),
            "max_rel_dist": float(rel.max()),
            "hit_rows_max_abs_dist": float(dd[h64].max()) if h64.any() else 0.0,
            "hit_rows_p99_abs_dist": float(np.percentile(dd[h64], 99)) if h64.any() else 0.0,
            f"share_beyond_{bound:g}": float(np.mean((rel if bound < 1e-3 else dd) > bound)),
            "max_abs_logit": float(dl.max()),
            "hit_mismatch_rate": float(np.mean(hit[clear] != (logit64[clear] > 0))),
            f"hit_mismatch_rate_outside_{band:g}": float(np.mean(hit[off] != (logit64[off] > 0))),
            "normal_rows": int(both.sum()), "normal_angle_deg_median": float(np.median(ang)),
            "normal_angle_deg_p99": float(np.percentile(ang, 99))}


def gpu_ray_set(torch, V, F, n, seed, sigma=0.05):
    """The labelled-ray recipe (half origins uniform on the unit sphere with uniform directions,
    half aimed at area-weighted surface points with a Gaussian angular jitter sigma), drawn on the
    device with torch for the 2^24-ray labelling workload; float32 (n, 3) origins and directions."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    dev = "cuda"

    def unit_dirs(m):
        z = 1.0 - 2.0 * torch.rand(m, device=dev, generator=g, dtype=torch.float64)
        a = 2.0 * math.pi * torch.rand(m, device=dev, generator=g, dtype=torch.float64)
        r = torch.sqrt(torch.clamp(1.0 - z * z, min=0.0))
        return torch.stack([r * torch.cos(a), r * torch.sin(a), z], 1)

    h = n // 2
    o1, w1 = unit_dirs(h), unit_dirs(h)
    Vt = torch.from_numpy(V).to(dev, torch.float64)
    Ft = torch.from_numpy(F.astype("int64")).to(dev)
    p0, p1, p2 = Vt[Ft[:, 0]], Vt[Ft[:, 1]], Vt[Ft[:, 2]]
    area = 0.5 * torch.linalg.norm(torch.cross(p1 - p0, p2 - p0, dim=1), dim=1)
    idx = torch.multinomial(area, n - h, replacement=True, generator=g)
    a = torch.rand(n - h, device=dev, generator=g, dtype=torch.float64)
    b = torch.rand(n - h, device=dev, generator=g, dtype=torch.float64)
    flip = a + b > 1.0
    a, b = torch.where(flip, 1.0 - a, a), torch.where(flip, 1.0 - b, b)
    pts = (1.0 - a - b)[:, None] * p0[idx] + a[:, None] * p1[idx] + b[:, None] * p2[idx]
    o2 = unit_dirs(n - h)
    w2 = torch.nn.functional.normalize(pts - o2, dim=1)
    helper = torch.where(w2[:, 2:3].abs() < 0.9, torch.tensor([[0.0, 0.0, 1.0]], device=dev, dtype=torch.float64),
                         torch.tensor([[1.0, 0.0, 0.0]], device=dev, dtype=torch.float64))
    t1 = torch.nn.functional.normalize(torch.cross(w2, helper, dim=1), dim=1)
    t2 = torch.cross(w2, t1, dim=1)
    gg = torch.randn(n - h, 2, device=dev, generator=g, dtype=torch.float64)
    w2 = torch.nn.functional.normalize(w2 + sigma * (gg[:, :1] * t1 + gg[:, 1:] * t2), dim=1)
    perm = torch.randperm(n, device=dev, generator=g)
    o = torch.cat([o1, o2])[perm]
    w = torch.nn.functional.normalize(torch.cat([w1, w2])[perm], dim=1)
    return o.float().contiguous(), w.float().contiguous()


def measured_peaks(P):
    """The throughput loops of ddf_measure_peaks on this device (TFLOP/s) and its SM count."""
    try:
        return P.measure_peaks()
    except Exception as e:   # the loops are a denominator only: report and fall back
        return {"error": str(e)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16", "fp8"])
    ap.add_argument("--ref-paths", type=int, default=2048)
    ap.add_argument("--no-oracle", action="store_true", help="skip the CPU oracle legs")
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--error-rays", type=int, default=1 << 20, help="rays of each query-error subset")
    ap.add_argument("--no-train", action="store_true", help="skip training the knot network and its rows")
    ap.add_argument("--no-rows", action="store_true", help="skip the labelling / training / grouped rows")
    ap.add_argument("--size", default="full", choices=["full", "small", "medium"],
                    help="small: 512 x 512 x 8 spp (2^21 paths) for profiler captures; medium: 512 x 512 x 32 spp "
                         "(2^23 paths: each bounce-1 launch's rays exceed the L2) for DRAM-traffic captures")
    ap.add_argument("--row", default=None, choices=["label", "sampler", "pov", "aov", "udf", "mesh_render", "train",
                                                   "grouped", "w512", "large"],
                    help="run only this row's workload (for profiler captures) and print it")
    args = ap.parse_args()
    if args.size == "small":
        WORKLOAD["spp"] = 8
    elif args.size == "medium":
        WORKLOAD["spp"] = 32
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2306_16142_gb300 as P
    from ddf_synth import default_camera, init_weights
    from paper_2306_16142_gb300.ddf import camera_struct
    peaks, peak_src = load_peaks()
    meas = measured_peaks(P)
    if args.row:
        print(json.dumps({"rows": other_rows(P, torch, np, peaks, meas, only=args.row, args=args, peak_src=peak_src)}),
              flush=True)
        return 0
    pool, jobs = None, {}
    if rank == 0 and not args.no_oracle:
        # the FP64 error jobs run in a spawned worker while the device works
        import concurrent.futures as cf
        import multiprocessing as mp
        keep = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
        nthr = str(max(1, (os.cpu_count() or 4) - 4))   # leave cores to the process that launches kernels
        os.environ["OPENBLAS_NUM_THREADS"] = os.environ["OMP_NUM_THREADS"] = nthr
        pool = cf.ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn"))
        pool.submit(int, 0).result()   # the worker starts (and reads its thread count) now
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    w = WORKLOAD
    E = 6 + 6 * w["in_freqs"]
    blob = init_weights(w["in_freqs"], w["hidden"], w["layers"], seed=w["seed"])
    prec = args.precision
    if prec == "auto":
        prec = "bf16"
    try:
        net = P.DDFNet(w["in_freqs"], w["hidden"], w["layers"], blob, prec)
    except P.DDFError:
        prec = "fp32"
        net = P.DDFNet(w["in_freqs"], w["hidden"], w["layers"], blob, prec)
    cam = default_camera(w["width"], w["height"], seed=1 + rank)
    img = torch.empty(w["height"], w["width"], device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        net.render(cam, w["spp"], w["bounces"], img)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    stats = net.render_stats(w["bounces"])

    # ---- timed region (device time, CUDA events on the launching stream)
    net.profile(True)
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    prof = net.profile_read()
    net.profile(False)
    ms = max_over_ranks(torch, ms, world)
    paths = w["width"] * w["height"] * w["spp"]
    value = whole_job_rate(paths, world, args.steps, ms)
    queries = sum(stats)
    queries_per_s = whole_job_rate(queries, world, args.steps, ms)

    # ---- dominant kernel roofline: the field query
    roof = query_roofline(stats, prof, ms, E, w["hidden"], w["layers"], prec, peaks, peak_src, meas, args.steps)
    if prec == "bf16":
        roof["traffic"] = query_traffic_per_bounce(stats, w["bounces"])
        roof["traffic_unit"] = ("bytes per bounce query (forward + normals launches), the per-row DRAM bytes of "
                                "one ncu capture of each kernel times this render's rows")

    # ---- wavefront kernels against HBM: algorithmic bytes per launch / measured launch time
    B = w["bounces"]
    shade_bytes = 0.0
    for b in range(B):
        live = stats[b]
        surv = stats[b + 1] if b + 1 < B else 0
        shade_bytes += 52.0 * live + 32.0 * surv + 4.0 * (live - surv)
    sh = prof["shade"]
    hbm = peaks["hbm_gbs"]
    shade_gbs = shade_bytes / B / (sh["ms"] / max(1, sh["launches"]) / 1e3) / 1e9
    rg = prof["raygen"]
    raygen_gbs = paths * 32.0 / (rg["ms"] / max(1, rg["launches"]) / 1e3) / 1e9
    wavefront_roofline = {
        "shade": {"bound": "hbm", "achieved": shade_gbs, "peak": hbm, "unit": "GB/s", "frac": shade_gbs / hbm,
                  "bytes": "52 B read per live ray + 32 B written per survivor + 4 B per terminated path"},
        "raygen": {"bound": "hbm", "achieved": raygen_gbs, "peak": hbm, "unit": "GB/s", "frac": raygen_gbs / hbm,
                   "bytes": "32 B of ray state written per path"},
        "time_share": {k: prof[k]["ms"] / ms for k in ("query", "shade", "raygen", "accumulate")}}

    # ---- end to end through the public call, image read back to pinned host memory
    host_img = torch.empty(w["height"], w["width"], pin_memory=True)
    cs = camera_struct(cam)
    for _ in range(2):
        net.render(cam, w["spp"], w["bounces"], img)
        host_img.copy_(img, non_blocking=True)
    torch.cuda.synchronize()
    e2e_steps = max(2, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        net.render(cam, w["spp"], w["bounces"], img)
        host_img.copy_(img, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": paths * world * e2e_steps / e2e_s, "unit": "samples/s",
           "h2d_bytes_per_step": int(np.dtype(np.uint8).itemsize * len(bytes(cs))),
           "d2h_bytes_per_step": int(host_img.numel() * 4)}

    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8e4m3"}[prec],
            "data": "synthetic",
            "config": {"workload": workload_name(w, trained=False), "precision": prec,
                       "paths_per_step": paths, "queries_per_step": queries, "queries_per_bounce": stats,
                       "l2": "no flush: ray state of one wave (2^24 paths, ~1.5 GB) exceeds the 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "queries_per_s": queries_per_s,
            "roofline": roof,
            "wavefront_roofline": wavefront_roofline,
            "e2e": e2e,
            # per wave: raygen, a forward launch per bounce, a normals launch per bounce but the
            # last, a shade launch per bounce, accumulate and the per-bounce count update
            "gpu_launches": int(args.steps * -(-paths // (1 << 24)) * (3 * w["bounces"] + 2)),
            "clocks": clocks}
    if rank == 0:
        line["peaks_measured_here"] = meas

    # ---- FP8 and FP32 paths on the same render
    nets = {prec: net}
    for other in ("fp8", "fp32"):
        if rank != 0 or prec != "bf16" or args.fp32_steps <= 0:
            break
        n2 = P.DDFNet(w["in_freqs"], w["hidden"], w["layers"], blob, other)
        nets[other] = n2
        n2.render(cam, w["spp"], w["bounces"], img)
        torch.cuda.synchronize()
        reps = max(2, args.fp32_steps) if other == "fp8" else args.fp32_steps
        n2.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            n2.render(cam, w["spp"], w["bounces"], img)
        e1.record(stream)
        torch.cuda.synchronize()
        pr2 = n2.profile_read()
        n2.profile(False)
        ms2 = e0.elapsed_time(e1)
        st2 = n2.render_stats(w["bounces"])
        line[f"{other}_path"] = {"value": paths * reps / (ms2 / 1e3), "unit": "samples/s",
                                 "queries_per_s": sum(st2) * reps / (ms2 / 1e3), "queries_per_bounce": st2,
                                 "roofline": query_roofline(st2, pr2, ms2, E, w["hidden"], w["layers"], other,
                                                            peaks, peak_src, meas, reps)}
    # ---- query errors of every precision against the oracle on 2^20 of the render's own rays
    if pool is not None:
        o_e, w_e, per_b = render_query_rays(P, torch, np, net, cam, w["spp"], w["bounces"], args.error_rays // 4, 13)
        to_e, tw_e = torch.from_numpy(o_e).cuda(), torch.from_numpy(w_e).cuda()
        outs = {}
        for k, nk in nets.items():
            r = nk.query(to_e, tw_e, normals=True)
            outs[k] = {kk: v.cpu().numpy() for kk, v in r.items()}
        hit_any = np.zeros(o_e.shape[0], bool)
        for r in outs.values():
            hit_any |= r["hit"].astype(bool)
        jobs["render"] = (pool.submit(oracle_query_job, blob, w["in_freqs"], w["hidden"], w["layers"], o_e, w_e,
                                      hit_any), outs, {"rays": int(o_e.shape[0]), "rays_per_bounce": per_b,
                                                       "source": "ddf_render_trace of random paths of the timed "
                                                                 "render (BF16), every bounce's query ray, this many "
                                                                 "of them drawn uniformly"})
    if rank == 0 and not args.no_train:
        # the knot network trained by the library, rendered the same way, with its query errors
        blob_t, train_info = train_knot_field(P, torch, np)
        trained = {"workload": workload_name(w, trained=True), "training": train_info}
        nets_t = {}
        for pr in ("bf16", "fp8", "fp32"):
            nt = P.DDFNet(w["in_freqs"], w["hidden"], w["layers"], blob_t, pr)
            nets_t[pr] = nt
            reps = 5 if pr != "fp32" else max(1, args.fp32_steps)
            nt.render(cam, w["spp"], w["bounces"], img)
            torch.cuda.synchronize()
            nt.profile(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                nt.render(cam, w["spp"], w["bounces"], img)
            e1.record(stream)
            torch.cuda.synchronize()
            prt = nt.profile_read()
            nt.profile(False)
            mst = e0.elapsed_time(e1)
            stt = nt.render_stats(w["bounces"])
            trained[pr] = {"samples_per_s": paths * reps / (mst / 1e3), "ms_per_render": mst / reps,
                           "queries_per_bounce": stt,
                           "roofline": query_roofline(stt, prt, mst, E, w["hidden"], w["layers"], pr, peaks,
                                                      peak_src, meas, reps)}
        if pool is not None:
            o_e, w_e, per_b = render_query_rays(P, torch, np, nets_t["bf16"], cam, w["spp"], w["bounces"],
                                                args.error_rays, 14)
            to_e, tw_e = torch.from_numpy(o_e).cuda(), torch.from_numpy(w_e).cuda()
            outs = {}
            for k, nk in nets_t.items():
                r = nk.query(to_e, tw_e, normals=True)
                outs[k] = {kk: v.cpu().numpy() for kk, v in r.items()}
            hit_any = np.zeros(o_e.shape[0], bool)
            for r in outs.values():
                hit_any |= r["hit"].astype(bool)
            jobs["trained"] = (pool.submit(oracle_query_job, blob_t, w["in_freqs"], w["hidden"], w["layers"], o_e,
                                           w_e, hit_any), outs,
                               {"rays": int(o_e.shape[0]), "rays_per_bounce": per_b,
                                "source": "ddf_render_trace of 2^20 random paths of the trained network's BF16 render, "
                                          "every bounce's query ray, 2^20 of them drawn uniformly; the oracle evaluates "
                                          "the FP32 master weights the training produced"})
        line["trained"] = trained
        del nets_t
    if rank == 0 and not args.no_rows:
        line["rows"] = other_rows(P, torch, np, peaks, meas, pool=pool, jobs=jobs, args=args, peak_src=peak_src)
    if pool is not None:
        bands = {"fp32": 1e-4, "bf16": 2e-2, "fp8": 6e-2}
        bounds = {"fp32": 1e-5, "bf16": 2e-2, "fp8": 6e-2}
        for key, (fut, outs, meta) in jobs.items():
            ref = fut.result()
            errs = {k: error_stats(v, ref, bands[k], bounds[k]) for k, v in outs.items()}
            if key == "render":
                line["query_error"] = dict(meta, **errs)
            elif key == "trained":
                line["trained"]["query_error"] = dict(meta, **errs)
            elif "rows" in line:
                line["rows"][key]["query_error"] = dict(meta, **errs)
        pool.shutdown()
        dt, nq = oracle_render_sample(w, blob, args.ref_paths)
        line["cpu_baseline"] = {"value": args.ref_paths / dt, "unit": "samples/s", "cores": cpu_threads(),
                                "kind": "oracle",
                                "sample": f"{args.ref_paths} random paths of the same render "
                                          f"({nq} field queries)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def query_roofline(stats, prof, ms, E, W, L, prec, peaks, peak_src, meas, renders=1):
    """Roofline of the field-query calls of `renders` profiled renders: algorithmic flops (forward
    on every live row, the reverse pass on the rows that hit and continue) over the calls' summed
    CUDA-event durations, against the measured peak of the precision."""
    B = len(stats)
    flops = 0.0
    for b in range(B):
        flops += stats[b] * fwd_flops(E, W, L)
        if b + 1 < B:
            flops += stats[b + 1] * bwd_flops(E, W, L)      # normals of the rows that hit
    q = prof["query"]
    achieved = flops * renders / (q["ms"] / 1e3) / 1e12
    if prec == "fp32":
        peak = max(meas.get("fp32_fma_tflops", 0.0), meas.get("fp32x2_fma_tflops", 0.0))
        src = "measured here: FP32 FMA loop (ddf_measure_peaks)"
        if not peak:
            import torch
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            src = "derived: SMs x 128 FP32 lanes x 2 x max SM clock"
        roof = {"bound": "alu", "peak_source": src}
    else:
        peak = peaks["bf16_tflops_sustained"] * (2.0 if prec == "fp8" else 1.0)
        roof = {"bound": "tensor",
                "peak_source": f"{peak_src} bf16 sustained" + (" x 2 (fp8 nominal ratio)" if prec == "fp8" else "")}
        key = "fp8_mma_tflops" if prec == "fp8" else "bf16_mma_tflops"
        if meas.get(key):
            roof["frac_of_mma_loop_here"] = achieved / meas[key]
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                 "kernel": "field query (fused MLP + Eq. 3 normal)", "time_share": q["ms"] / ms if ms > 0 else None})
    return roof


def _time(torch, fn, reps, stream=None):
    """Device time per call of fn (CUDA events on the current stream), after 2 warm-up calls."""
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def fp32_lane_peak(meas, peaks, torch):
    """FP32 lane operations per second: the measured FMA loop (an FMA or one lane of a packed FP32x2
    FMA is one operation; the packed form issues half the instructions at the same lane rate), else
    SMs x 128 lanes x the maximum SM clock."""
    m = max(meas.get("fp32_fma_tflops", 0.0), meas.get("fp32x2_fma_tflops", 0.0))
    if m:
        return m * 1e12 / 2.0, "measured here (ddf_measure_peaks FMA loops)"
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6, "derived: SMs x 128 lanes x max SM clock"


def other_rows(P, torch, np, peaks, meas, only=None, pool=None, jobs=None, args=None, peak_src="measured"):
    """The other hot-path rows on their own workloads: ray labelling (2^20 training rays x 8,192-
    triangle knot), the training-set samplers, depth / normal images, the mesh path tracer, the UDF,
    the training step (batch 65,536, 78 -> 256 x 8 -> 2; BF16 tensor-core and FP32), the grouped
    16-object BF16 query replayed from a CUDA graph (widths 128 / 256 / 512, ray counts log-uniform
    on [1e3, 1e6]), the width-512 query and the full large render with its labelling workload.
    only: one row name (the others are skipped). pool / jobs: the spawned oracle worker and the
    error jobs submitted to it (the large render adds one)."""
    from ddf_synth import default_camera, init_weights, labelled_ray_set, torus_knot
    rows = {}
    want = lambda name: only is None or only == name
    alu_peak, alu_src = fp32_lane_peak(meas, peaks, torch)
    V, F = torus_knot(3, 2, 0.08, 256, 16)
    mesh = P.DDFMesh(V, F)
    if want("label") or want("train"):
        o, w = labelled_ray_set(V, F, 1 << 20, seed=11)
        to, tw = torch.from_numpy(o).cuda(), torch.from_numpy(w).cuda()
    # ---- a8 labelling
    if want("label"):
        out = mesh.label(to, tw)
        # the sweep over all faces (FP32 issue-bound)
        mesh.set_accel("none")
        sec = _time(torch, lambda: mesh.label(to, tw, out), 5)
        st = mesh.stats()
        tests = o.shape[0] * F.shape[0]
        sweep = {"ms": sec * 1e3, "rays_per_s": o.shape[0] / sec, "tests_per_s": tests / sec,
                 "fp64_retests_per_ray": st["retests"] / o.shape[0],
                 "roofline": {"bound": "alu", "achieved": tests / sec * 34 / 1e12,
                              "peak": alu_peak / 1e12, "unit": "T FP32 lane-ops/s",
                              "frac": tests / sec * 34 / alu_peak,
                              "peak_source": alu_src,
                              "note": "34 FP32 lane operations per filter test (count of the hot loop; the "
                                      "thread's two rays run as the two lanes of packed FP32x2 instructions, "
                                      "each lane one operation: the measured packed FMA rate equals the "
                                      "scalar one per lane)"}}
        # the hierarchy (the default): the same labels, a few dozen node visits and face tests per ray
        mesh.set_accel("bvh")
        secb = _time(torch, lambda: mesh.label(to, tw, out), 5)
        bs = mesh.bvh_stats()
        stb = mesh.stats()
        rows["label"] = {"workload": "2^20 rays (half uniform, half surface-aimed, sigma 0.05 rad) x 8,192-triangle "
                                     "(3,2) knot",
                         "rays_per_s": o.shape[0] / secb, "ms": secb * 1e3, "accel": "bvh",
                         "bvh": {"nodes": bs["nodes"], "depth": bs["depth"],
                                 "node_visits_per_ray": bs["visits"] / o.shape[0],
                                 "face_tests_per_ray": bs["face_tests"] / o.shape[0],
                                 "fp64_retests_per_ray": stb["retests"] / o.shape[0],
                                 "node_bytes_per_s": bs["visits"] * 64 / secb,
                                 "note": "64-byte two-box nodes and 48-byte faces, all resident in L2: a "
                                         "latency-bound traversal with no HBM roofline"},
                         "sweep": sweep, "speedup_vs_sweep": sec / secb}
    # ---- the surface-marching training-set sampler (Sec. 5.2), Table 2's smallest setting
    if want("sampler"):
        s = 10
        C = F.shape[0] * s * s
        first = mesh.sample_surface(s, s, s, 1e-4, 21)
        buf = P.DDFMesh.sample_buffers(first["count"])
        sec = _time(torch, lambda: mesh.sample_surface(s, s, s, 1e-4, 21, out=buf), 2)
        mesh.set_accel("none")
        sec_sweep = _time(torch, lambda: mesh.sample_surface(s, s, s, 1e-4, 21, out=buf), 1)
        mesh.set_accel("bvh")
        n = first["count"]
        kinds = np.bincount((first["key"] % 4).cpu().numpy(), minlength=4)
        rays = C + 2 * int(kinds[1])      # candidates + two Eq. 12 rays per march point of a missing one
        tests = rays * F.shape[0]
        rows["sampler"] = {"workload": "s_fc = s_dr = s_p = 10 on the 8,192-triangle (3,2) knot: 819,200 candidate "
                                       "rays, odd-even parity, marching, Eq. 12 rays of the missing candidates",
                           "samples": n, "samples_per_s": n / sec, "ms": sec * 1e3, "accel": "bvh",
                           "kinds": [int(x) for x in kinds], "labelled_rays": rays,
                           "sweep": {"ms": sec_sweep * 1e3,
                                     "roofline": {"bound": "alu", "achieved": tests / sec_sweep * 34 / 1e12,
                                                  "peak": alu_peak / 1e12, "unit": "T FP32 lane-ops/s",
                                                  "frac": tests / sec_sweep * 34 / alu_peak,
                                                  "note": "the labeller's filter tests over the whole call "
                                                          "(allocation, two host scans and the other kernels "
                                                          "included)"}}}
        del first, buf
    # ---- the point-of-view sampling of Sec. 6: 10 x 5 cameras, 256 x 256 films
    if want("pov"):
        n = 50 * 256 * 256
        pbuf = mesh.sample_pov(10, 5, 256)
        sec = _time(torch, lambda: mesh.sample_pov(10, 5, 256, out=pbuf), 3)
        mesh.set_accel("none")
        sec_sweep = _time(torch, lambda: mesh.sample_pov(10, 5, 256, out=pbuf), 2)
        mesh.set_accel("bvh")
        tests = n * F.shape[0]
        rows["pov"] = {"workload": "10 x 5 cameras at distance 2.5, 30 deg field of view, 256 x 256 pixels each "
                                   "(3,276,800 rays) labelled against the 8,192-triangle (3,2) knot",
                       "rays_per_s": n / sec, "ms": sec * 1e3, "accel": "bvh", "hits": int(pbuf["hit"].sum().item()),
                       "sweep": {"ms": sec_sweep * 1e3,
                                 "roofline": {"bound": "alu", "achieved": tests / sec_sweep * 34 / 1e12,
                                              "peak": alu_peak / 1e12, "unit": "T FP32 lane-ops/s",
                                              "frac": tests / sec_sweep * 34 / alu_peak,
                                              "note": "the labeller's filter tests; ray generation included"}}}
        del pbuf
    # ---- depth + normal images (Fig. 3 / 4) from the field and from the mesh (Fig. 5's comparison)
    if want("aov"):
        w_ = WORKLOAD
        camA = default_camera(1920, 1080, seed=1)
        netA = P.DDFNet(w_["in_freqs"], w_["hidden"], w_["layers"],
                        init_weights(w_["in_freqs"], w_["hidden"], w_["layers"], seed=w_["seed"]), "bf16")
        secA = _time(torch, lambda: netA.render_aov(camA), 5)
        npx = 1920 * 1080
        mesh_ms = {}
        for label_, (Vm, Fm) in (("8,192-triangle knot", (V, F)),
                                 ("131,072-triangle knot", torus_knot(3, 2, 0.08, 1024, 64))):
            mA = P.DDFMesh(Vm, Fm)
            mesh_ms[label_ + ", bvh"] = _time(torch, lambda: mA.render_aov(camA), 3) * 1e3
            mA.set_accel("none")
            mesh_ms[label_ + ", all faces"] = _time(torch, lambda: mA.render_aov(camA), 1) * 1e3
            del mA
        rows["aov"] = {"workload": "1920 x 1080 depth + normal images, one ray per pixel: the BF16 field "
                                   "(78 -> 256 x 8 -> 2) against casting the same rays on meshes (through the "
                                   "hierarchy, and against all faces)",
                       "field_ms": secA * 1e3, "field_rays_per_s": npx / secA, "mesh_ms": mesh_ms}
        del netA
    # ---- the path tracer with the mesh in place of the field (Fig. 5's "without DDF"), same render
    if want("mesh_render"):
        w_ = WORKLOAD
        camM = default_camera(w_["width"], w_["height"], seed=1)
        imgM = torch.empty(w_["height"], w_["width"], device="cuda")
        secM = _time(torch, lambda: mesh.render(camM, w_["spp"], w_["bounces"], imgM), 3)
        nS = w_["width"] * w_["height"] * w_["spp"]
        rows["mesh_render"] = {"workload": f"{w_['width']} x {w_['height']} x {w_['spp']} spp, <= {w_['bounces']} bounces "
                                           "(the headline render) with the 8,192-triangle knot cast through the BVH "
                                           "in place of the field",
                               "samples_per_s": nS / secM, "ms": secM * 1e3,
                               "note": "allocation of the wavefront buffers included (the call is synchronous)"}
    # ---- the UDF of Eq. 4: the minimum over 256 directions for 65,536 points
    if want("udf"):
        from ddf_synth import fibonacci_directions
        w_ = WORKLOAD
        netU = P.DDFNet(w_["in_freqs"], w_["hidden"], w_["layers"],
                        init_weights(w_["in_freqs"], w_["hidden"], w_["layers"], seed=w_["seed"]), "bf16")
        gU = torch.Generator(device="cuda").manual_seed(17)
        pts = torch.randn(65536, 3, device="cuda", generator=gU)
        pts = pts / pts.norm(dim=1, keepdim=True) * torch.rand(65536, 1, device="cuda", generator=gU)
        dirsU = torch.from_numpy(fibonacci_directions(256)).cuda()
        secU = _time(torch, lambda: netU.udf(pts, dirsU), 3)
        q = 65536 * 256
        fq = 2.0 * ((6 + 6 * w_["in_freqs"]) * w_["hidden"] + (w_["layers"] - 1) * w_["hidden"] ** 2 + 2 * w_["hidden"])
        peak = peaks["bf16_tflops_sustained"]
        rows["udf"] = {"workload": "UDF (Eq. 4) of 65,536 points in the unit ball over 256 Fibonacci directions "
                                   "(16.8M queries), BF16 78 -> 256 x 8 -> 2",
                       "points_per_s": 65536 / secU, "queries_per_s": q / secU, "ms": secU * 1e3,
                       "roofline": {"bound": "tensor", "achieved": fq * q / secU / 1e12, "peak": peak,
                                    "unit": "TFLOP/s", "frac": fq * q / secU / 1e12 / peak,
                                    "note": "the forward flops of the queries over the whole call (ray build, "
                                            "min reduction and allocation included)"}}
        del netU
    # ---- a9 training step: BF16 tensor-core GEMMs (FP32 accumulate, FP32 masters), and the FP32 path
    if want("train"):
        Fq, Wd, Ld = 12, 256, 8
        n = 65536
        lab = mesh.label(to[:n].contiguous(), tw[:n].contiguous())
        dgt, hgt = lab["dist"].clone(), lab["hit"].clone()
        tsub, wsub = to[:n].contiguous(), tw[:n].contiguous()
        loss = torch.empty((), device="cuda")
        E = 6 + 6 * Fq
        macs = E * Wd + (Ld - 1) * Wd * Wd + 2 * Wd
        for prec in ("bf16", "fp32") if only is None else ("bf16",):
            net = P.DDFNet(Fq, Wd, Ld, init_weights(Fq, Wd, Ld, seed=2), prec)
            sec = _time(torch, lambda: net.train_step(tsub, wsub, dgt, hgt, lr=1e-4, loss=loss),
                        10 if prec == "bf16" else 3)
            net.device_status()
            if prec == "bf16":
                flop = 2.0 * macs * n * 3     # forward, dgrad, wgrad (activations kept, no recompute)
                peak = peaks["bf16_tflops_sustained"]
                rows["train_step"] = {"workload": "batch 65,536 labelled rays, 78 -> 256 x 8 -> 2, L1 + BCE, Adam; "
                                                  "BF16 tcgen05 GEMMs, FP32 accumulate and masters",
                                      "ms": sec * 1e3, "samples_per_s": n / sec, "loss": float(loss.item()),
                                      "roofline": {"bound": "tensor", "achieved": flop / sec / 1e12, "peak": peak,
                                                   "unit": "TFLOP/s", "frac": flop / sec / 1e12 / peak}}
            else:
                flop = 2.0 * macs * n * 4     # forward, recomputed forward, dgrad, wgrad
                fp32_peak = 2.0 * alu_peak
                rows["train_step_fp32"] = {"workload": "the same step on the FP32 SIMT GEMMs",
                                           "ms": sec * 1e3, "samples_per_s": n / sec,
                                           "roofline": {"bound": "alu", "achieved": flop / sec / 1e12,
                                                        "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                                                        "frac": flop / sec / fp32_peak}}
            del net
    # ---- a10 grouped query (16 objects, widths 128 / 256 / 512, 4-8 layers)
    if want("grouped"):
        rng = np.random.default_rng(14)
        specs = [(12, (128, 256, 512)[i % 3], 4 + (7 * i) % 5, 100 + i) for i in range(16)]
        nets = [P.DDFNet(Fq2, W2, L2, init_weights(Fq2, W2, L2, seed=s2), "bf16") for Fq2, W2, L2, s2 in specs]
        counts = np.floor(10 ** (3 + 3 * rng.random(16))).astype(np.int64)
        off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        tot = int(off[-1])
        g = torch.Generator(device="cuda").manual_seed(15)
        go = torch.randn(tot, 3, device="cuda", generator=g)
        go = go / go.norm(dim=1, keepdim=True) * torch.rand(tot, 1, device="cuda", generator=g)
        gw = torch.randn(tot, 3, device="cuda", generator=g)
        gw = gw / gw.norm(dim=1, keepdim=True)
        toff = torch.from_numpy(off).cuda()
        grp = P.DDFGroup(nets)
        gout = grp._out(tot, "cuda")
        cfg = grp.autotune(toff, go, gw, gout, reps=2)
        grp.capture(toff, go, gw, gout)
        sec = _time(torch, grp.replay, 10)
        grp.status()
        flop = sum(2.0 * ((6 + 6 * f) * W2 + (L2 - 1) * W2 * W2 + 2 * W2) * c
                   for (f, W2, L2, _), c in zip(specs, counts))
        peak = peaks["bf16_tflops_sustained"]
        by_w = {str(W2): int(sum(c for (_, ww, _, _), c in zip(specs, counts) if ww == W2)) for W2 in (128, 256, 512)}
        rows["grouped_query"] = {"workload": "16 BF16 networks (widths 128 / 256 / 512, 4-8 layers, 12-frequency "
                                             "encoding), ray counts log-uniform on [1e3, 1e6], one CUDA-graph replay "
                                             "per bounce",
                                 "rays": tot, "rays_per_width": by_w, "queries_per_s": tot / sec, "ms": sec * 1e3,
                                 "launch_shapes": cfg,
                                 "roofline": {"bound": "tensor", "achieved": flop / sec / 1e12, "peak": peak,
                                              "unit": "TFLOP/s", "frac": flop / sec / 1e12 / peak,
                                              "note": "algorithmic forward flops of all objects over one replay"}}
        del grp, nets
    # ---- width-512 network (102 -> 512 x 8 -> 2) queries, BF16 and FP8
    if want("w512"):
        F5, W5, L5 = 16, 512, 8
        blob5 = init_weights(F5, W5, L5, seed=5)
        nq = 1 << 22
        g5 = torch.Generator(device="cuda").manual_seed(16)
        qo = torch.randn(nq, 3, device="cuda", generator=g5)
        qo = qo / qo.norm(dim=1, keepdim=True) * torch.rand(nq, 1, device="cuda", generator=g5)
        qw = torch.randn(nq, 3, device="cuda", generator=g5)
        qw = qw / qw.norm(dim=1, keepdim=True)
        f5 = 2.0 * ((6 + 6 * F5) * W5 + (L5 - 1) * W5 * W5 + 2 * W5)
        for pr in ("bf16", "fp8"):
            n5 = P.DDFNet(F5, W5, L5, blob5, pr)
            qout = n5.query(qo, qw)
            sec = _time(torch, lambda: n5.query(qo, qw, out=qout), 3)
            peak = peaks["bf16_tflops_sustained"] * (2.0 if pr == "fp8" else 1.0)
            rows[f"query_w512_{pr}"] = {
                "workload": f"2^22 queries, 102 -> 512 x 8 -> 2, {pr.upper()}, no normals",
                "queries_per_s": nq / sec, "ms": sec * 1e3,
                "roofline": {"bound": "tensor", "achieved": f5 * nq / sec / 1e12, "peak": peak, "unit": "TFLOP/s",
                             "frac": f5 * nq / sec / 1e12 / peak,
                             "peak_source": "bf16 sustained" + (" x 2 (fp8 nominal ratio)" if pr == "fp8" else "")}}
            del n5
    # ---- the large render: 1920 x 1080 x 256 spp, <= 8 bounces, 102 -> 512 x 8 -> 2, FP32 / BF16 / FP8,
    #      and 2^24 labelled rays against the 131,072-face knot
    if want("large"):
        Lw = LARGE
        F5, W5, L5 = Lw["in_freqs"], Lw["hidden"], Lw["layers"]
        E5 = 6 + 6 * F5
        blob5 = init_weights(F5, W5, L5, seed=Lw["seed"])
        cam5 = default_camera(Lw["width"], Lw["height"], seed=1)
        img5 = torch.empty(Lw["height"], Lw["width"], device="cuda")
        host5 = torch.empty(Lw["height"], Lw["width"], pin_memory=True)
        paths5 = Lw["width"] * Lw["height"] * Lw["spp"]
        big = {"workload": f"{Lw['width']} x {Lw['height']} x {Lw['spp']} spp ({paths5:,} paths in "
                           f"{-(-paths5 // (1 << 24))} waves), <= {Lw['bounces']} bounces, {E5} -> {W5} x {L5} -> 2 "
                           f"DDF MLP (seeded weights)"}
        nets5 = {}
        for pr in ("bf16", "fp8"):
            n5 = P.DDFNet(F5, W5, L5, blob5, pr)
            nets5[pr] = n5
            n5.render(cam5, Lw["spp"], Lw["bounces"], img5)
            torch.cuda.synchronize()
            n5.profile(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            n5.render(cam5, Lw["spp"], Lw["bounces"], img5)
            e1.record()
            torch.cuda.synchronize()
            pr5 = n5.profile_read()
            n5.profile(False)
            ms5 = e0.elapsed_time(e1)
            st5 = n5.render_stats(Lw["bounces"])
            t0 = time.perf_counter()
            n5.render(cam5, Lw["spp"], Lw["bounces"], img5)
            host5.copy_(img5, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            e2e5 = time.perf_counter() - t0
            n5.device_status()
            big[pr] = {"samples_per_s": paths5 / (ms5 / 1e3), "ms": ms5, "queries_per_bounce": st5,
                       "queries_per_s": sum(st5) / (ms5 / 1e3),
                       "e2e": {"value": paths5 / e2e5, "unit": "samples/s", "h2d_bytes_per_step": 64,
                               "d2h_bytes_per_step": int(host5.numel() * 4)},
                       "roofline": query_roofline(st5, pr5, ms5, E5, W5, L5, pr, peaks, peak_src, meas)}
        # FP32 SIMT on one 8-spp wave of the same camera (1/32 of the paths), timed once after a warm-up
        n32 = P.DDFNet(F5, W5, L5, blob5, "fp32")
        nets5["fp32"] = n32
        sec32 = _time(torch, lambda: n32.render(cam5, 8, Lw["bounces"], img5), 1)
        big["fp32"] = {"samples_per_s": Lw["width"] * Lw["height"] * 8 / sec32, "ms": sec32 * 1e3,
                       "sample": "one 8-spp wave of the same camera (16.6M paths, 1/32 of the render)",
                       "queries_per_bounce": n32.render_stats(Lw["bounces"])}
        if pool is not None and jobs is not None:
            n_err = args.error_rays if args is not None else 1 << 20
            o_e, w_e, per_b = render_query_rays(P, torch, np, nets5["bf16"], cam5, Lw["spp"], Lw["bounces"], n_err, 15)
            to_e, tw_e = torch.from_numpy(o_e).cuda(), torch.from_numpy(w_e).cuda()
            outs = {}
            for k, nk in nets5.items():
                r = nk.query(to_e, tw_e, normals=True)
                outs[k] = {kk: v.cpu().numpy() for kk, v in r.items()}
            hit_any = np.zeros(o_e.shape[0], bool)
            for r in outs.values():
                hit_any |= r["hit"].astype(bool)
            jobs["large_render"] = (pool.submit(oracle_query_job, blob5, F5, W5, L5, o_e, w_e, hit_any), outs,
                                    {"rays": int(o_e.shape[0]), "rays_per_bounce": per_b,
                                     "source": "ddf_render_trace of 2^20 random paths of the BF16 render, every "
                                               "bounce's query ray, 2^20 of them drawn uniformly"})
        del nets5, n32
        # labelling: 2^24 rays (half uniform, half surface-aimed) x the 131,072-face knot
        V5, T5 = torus_knot(3, 2, 0.08, 1024, 64)
        m5 = P.DDFMesh(V5, T5)
        lo, lw = gpu_ray_set(torch, V5, T5, 1 << 24, seed=15)
        lab_b = m5.label(lo, lw)
        secb = _time(torch, lambda: m5.label(lo, lw, lab_b), 3)
        bs, stb = m5.bvh_stats(), m5.stats()
        m5.set_accel("none")
        lab_s = {k: torch.empty_like(v) for k, v in lab_b.items()}
        t0 = time.perf_counter()
        m5.label(lo, lw, lab_s)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        sts = m5.stats()
        same = bool(torch.equal(lab_b["tri"], lab_s["tri"]) and torch.equal(lab_b["hit"], lab_s["hit"])
                    and torch.equal(lab_b["dist"], lab_s["dist"]))
        tests = float(1 << 24) * T5.shape[0]
        big["label"] = {"workload": "2^24 rays (half uniform on the bounding sphere, half aimed at the surface with "
                                    "0.05 rad of jitter) x the 131,072-face (3,2) knot",
                        "bvh": {"ms": secb * 1e3, "rays_per_s": (1 << 24) / secb,
                                "node_visits_per_ray": bs["visits"] / (1 << 24),
                                "face_tests_per_ray": bs["face_tests"] / (1 << 24),
                                "fp64_retests_per_ray": stb["retests"] / (1 << 24),
                                "fp64_final_evals_per_ray": stb["finals"] / (1 << 24)},
                        "all_faces": {"ms": secs * 1e3, "tests_per_s": tests / secs,
                                      "fp64_retests_per_ray": sts["retests"] / (1 << 24),
                                      "roofline": {"bound": "alu", "achieved": tests / secs * 34 / 1e12,
                                                   "peak": alu_peak / 1e12, "unit": "T FP32 lane-ops/s",
                                                   "frac": tests / secs * 34 / alu_peak, "peak_source": alu_src}},
                        "labels_identical": same,
                        "hit_fraction": float(lab_b["hit"].float().mean().item())}
        rows["large_render"] = big
        del m5, lo, lw, lab_b, lab_s
    return rows


if __name__ == "__main__":
    sys.exit(main())
