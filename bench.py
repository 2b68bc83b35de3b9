"""Benchmark of the DDF hot path on GB300.

One step = one full render of the single-object workload (the modified path tracer of the
paper's Sec. 1 / Fig. 1): 512 x 512 pixels x 64 samples, at most 4 bounces, a 78 -> 256 x 8 -> 2
network (12-frequency encoding) with seeded weights, one wave of 2^24 paths: camera rays, one
batched field query per bounce (distance, hit, Eq. 3 normal), shading + compaction, per-pixel
accumulation - every step in libddf.so's kernels.

Prints ONE JSON line (rank 0): samples/s over the timed steps (device time, CUDA events, max over
ranks), the dominant kernel's roofline, the end-to-end figure through the public API with the
image read back to pinned host memory, the FP64 oracle timed on the host cores on a bounded
sample, SM clocks sampled during the timed region, and the query error against the oracle.

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


def workload_name(w):
    E = 6 + 6 * w["in_freqs"]
    return (f"single-object render {w['width']}x{w['height']} x {w['spp']} spp, <= {w['bounces']} bounces, "
            f"{E}->{w['hidden']}x{w['layers']}->2 DDF MLP (seeded weights)")


def fwd_flops(E, W, L):
    return 2.0 * (E * W + (L - 1) * W * W + 2 * W)


def bwd_flops(E, W, L):
    # reverse pass to the input for a hit row: W x W per hidden layer after the first, W x E last
    return 2.0 * ((L - 1) * W * W + W * E)


# ncu-measured DRAM traffic of the BF16 query kernels (mlp_pair_kernel<256> forward and
# mlp_tc_kernel<256,1> normals, the 7 launches of one 512 x 512 x 64 spp render); to be
# re-measured whenever the kernels change.
QUERY_DRAM_BYTES_PER_RENDER = 757.8e6


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
            "config": {"workload": workload_name(w), "parallelism": "host cores (numpy FP64 oracle)"},
            "queries_per_s": sum(nqs) / tot,
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{n_paths} random paths of the {w['width']}x{w['height']}x{w['spp']} "
                                       f"render per step"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    ap.add_argument("--no-rows", action="store_true", help="skip the labelling / training / grouped rows")
    ap.add_argument("--size", default="full", choices=["full", "small"],
                    help="small: 512 x 512 x 8 spp (2^21 paths) for profiler captures")
    ap.add_argument("--row", default=None, choices=["label", "sampler", "pov", "aov", "udf", "mesh_render", "train",
                                                   "grouped", "w512"],
                    help="run only this row's workload (for profiler captures) and print it")
    args = ap.parse_args()
    if args.size == "small":
        WORKLOAD["spp"] = 8
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
    if args.row:
        print(json.dumps({"rows": other_rows(P, torch, np, load_peaks()[0], only=args.row)}), flush=True)
        return 0

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
    Wd, Ld = w["hidden"], w["layers"]
    flops = 0.0
    for b in range(w["bounces"]):
        flops += stats[b] * fwd_flops(E, Wd, Ld)
        if b + 1 < w["bounces"]:
            flops += stats[b + 1] * bwd_flops(E, Wd, Ld)      # normals of the rows that hit
    q = prof["query"]
    q_launch_ms = q["ms"] / max(1, q["launches"])
    flops_per_launch = flops / w["bounces"]
    achieved = flops_per_launch / (q_launch_ms / 1e3) / 1e12
    peaks, peak_src = load_peaks()
    if prec == "fp32":
        # FP32 SIMT: 152 SMs x 128 FMA lanes x 2 flop x max SM clock
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz"}
    else:
        peak = peaks["bf16_tflops_sustained"] * (2.0 if prec == "fp8" else 1.0)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": f"{peak_src} bf16 sustained" + (" x 2 (fp8 nominal ratio)" if prec == "fp8" else "")}
        if prec == "bf16" and args.size == "full":
            # DRAM bytes (read + write) of the query kernels of one bench render, measured by ncu
            # (dram__bytes_read.sum + dram__bytes_write.sum, one pass, full size; summary in
            # profiles/bf16_query_render512x512.md), per bounce query like `achieved`
            roof["traffic"] = QUERY_DRAM_BYTES_PER_RENDER / w["bounces"]
            roof["traffic_unit"] = "bytes per bounce query (forward + normals launches)"
    roof["kernel"] = "field query (fused MLP + Eq. 3 normal)"
    roof["time_share"] = q["ms"] / ms if ms > 0 else None

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
    raygen_gbs = paths * (32.0 + 4.0 * 0) / (rg["ms"] / max(1, rg["launches"]) / 1e3) / 1e9
    wavefront_roofline = {
        "shade": {"bound": "hbm", "achieved": shade_gbs, "peak": hbm, "unit": "GB/s", "frac": shade_gbs / hbm,
                  "bytes": "52 B read per live ray + 32 B written per survivor + 4 B per terminated path"},
        "raygen": {"bound": "hbm", "achieved": raygen_gbs, "peak": hbm, "unit": "GB/s", "frac": raygen_gbs / hbm,
                   "bytes": "32 B of ray state written per path"}}

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
            "config": {"workload": workload_name(w), "precision": prec, "paths_per_step": paths,
                       "queries_per_step": queries, "queries_per_bounce": stats,
                       "l2": "no flush: ray state of one wave (2^24 paths, ~1.5 GB) exceeds the 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "queries_per_s": queries_per_s,
            "roofline": roof,
            "wavefront_roofline": wavefront_roofline,
            "e2e": e2e,
            "gpu_launches": int(sum(v["launches"] for v in prof.values()) + args.steps * 2),
            "clocks": clocks}

    # ---- FP8 path on the same render, with its query error
    if rank == 0 and prec == "bf16" and args.fp32_steps > 0:
        net8 = P.DDFNet(w["in_freqs"], w["hidden"], w["layers"], blob, "fp8")
        net8.render(cam, w["spp"], w["bounces"], img)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(max(2, args.fp32_steps)):
            net8.render(cam, w["spp"], w["bounces"], img)
        e1.record(stream)
        torch.cuda.synchronize()
        line["fp8_path"] = {"value": paths * max(2, args.fp32_steps) / (e0.elapsed_time(e1) / 1e3),
                            "unit": "samples/s"}
        if not args.no_oracle:
            line["fp8_path"]["query_error"] = query_error(P, net8, blob, w)
    # ---- FP32 path beside the tensor-core path, and the oracle
    if rank == 0 and prec != "fp32" and args.fp32_steps > 0:
        net32 = P.DDFNet(w["in_freqs"], w["hidden"], w["layers"], blob, "fp32")
        net32.render(cam, w["spp"], w["bounces"], img)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp32_steps):
            net32.render(cam, w["spp"], w["bounces"], img)
        e1.record(stream)
        torch.cuda.synchronize()
        line["fp32_path"] = {"value": paths * args.fp32_steps / (e0.elapsed_time(e1) / 1e3),
                             "unit": "samples/s"}
    if rank == 0 and not args.no_rows:
        line["rows"] = other_rows(P, torch, np, peaks)
    if rank == 0 and not args.no_oracle:
        line["query_error"] = query_error(P, net, blob, w)
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


def other_rows(P, torch, np, peaks, only=None):
    """The other hot-path rows on their own workloads: ray labelling (2^20 training rays x 8,192-
    triangle knot), the training step (batch 65,536, 78 -> 256 x 8 -> 2; BF16 tensor-core and FP32),
    the grouped 16-object BF16 query replayed from a CUDA graph (ray counts log-uniform on
    [1e3, 1e6]), the width-512 query and one wave of the large render. only: one of
    label / train / grouped / w512 (the others are skipped)."""
    from ddf_synth import default_camera, init_weights, labelled_ray_set, torus_knot
    rows = {}
    want = lambda name: only is None or only == name
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
        alu_peak = 152 * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6      # FP32 lane-instructions / s
        sweep = {"ms": sec * 1e3, "rays_per_s": o.shape[0] / sec, "tests_per_s": tests / sec,
                 "fp64_retests_per_ray": st["retests"] / o.shape[0],
                 "roofline": {"bound": "alu", "achieved": tests / sec * 34 / 1e12,
                              "peak": alu_peak / 1e12, "unit": "T FP32-instr/s",
                              "frac": tests / sec * 34 / alu_peak,
                              "note": "34 FP32 operations per filter test (count of the hot loop; the "
                                      "thread's two rays run as the lanes of packed FP32 pairs)"}}
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
        alu_peak = 152 * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
        rows["sampler"] = {"workload": "s_fc = s_dr = s_p = 10 on the 8,192-triangle (3,2) knot: 819,200 candidate "
                                       "rays, odd-even parity, marching, Eq. 12 rays of the missing candidates",
                           "samples": n, "samples_per_s": n / sec, "ms": sec * 1e3, "accel": "bvh",
                           "kinds": [int(x) for x in kinds], "labelled_rays": rays,
                           "sweep": {"ms": sec_sweep * 1e3,
                                     "roofline": {"bound": "alu", "achieved": tests / sec_sweep * 34 / 1e12,
                                                  "peak": alu_peak / 1e12, "unit": "T FP32-instr/s",
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
        alu_peak = 152 * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
        rows["pov"] = {"workload": "10 x 5 cameras at distance 2.5, 30 deg field of view, 256 x 256 pixels each "
                                   "(3,276,800 rays) labelled against the 8,192-triangle (3,2) knot",
                       "rays_per_s": n / sec, "ms": sec * 1e3, "accel": "bvh", "hits": int(pbuf["hit"].sum().item()),
                       "sweep": {"ms": sec_sweep * 1e3,
                                 "roofline": {"bound": "alu", "achieved": tests / sec_sweep * 34 / 1e12,
                                              "peak": alu_peak / 1e12, "unit": "T FP32-instr/s",
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
                fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6
                rows["train_step_fp32"] = {"workload": "the same step on the FP32 SIMT GEMMs",
                                           "ms": sec * 1e3, "samples_per_s": n / sec,
                                           "roofline": {"bound": "alu", "achieved": flop / sec / 1e12,
                                                        "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                                                        "frac": flop / sec / fp32_peak}}
            del net
    # ---- a10 grouped query (16 objects, widths 128 / 256, 4-8 layers)
    if want("grouped"):
        rng = np.random.default_rng(14)
        specs = [(12, 128 if i % 2 == 0 else 256, 4 + (i % 5), 100 + i) for i in range(16)]
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
        rows["grouped_query"] = {"workload": "16 BF16 networks (widths 128/256, 4-8 layers, 12-frequency encoding), "
                                             "ray counts log-uniform on [1e3, 1e6], one CUDA-graph replay per bounce",
                                 "rays": tot, "queries_per_s": tot / sec, "ms": sec * 1e3,
                                 "launch_shapes": cfg,
                                 "roofline": {"bound": "tensor", "achieved": flop / sec / 1e12, "peak": peak,
                                              "unit": "TFLOP/s", "frac": flop / sec / 1e12 / peak}}
    # ---- width-512 network (102 -> 512 x 8 -> 2) queries and one wave of the large render
    if want("w512"):
        F5, W5, L5 = 16, 512, 8
        blob5 = init_weights(F5, W5, L5, seed=5)
        n5 = P.DDFNet(F5, W5, L5, blob5, "bf16")
        nq = 1 << 22
        g5 = torch.Generator(device="cuda").manual_seed(16)
        qo = torch.randn(nq, 3, device="cuda", generator=g5)
        qo = qo / qo.norm(dim=1, keepdim=True) * torch.rand(nq, 1, device="cuda", generator=g5)
        qw = torch.randn(nq, 3, device="cuda", generator=g5)
        qw = qw / qw.norm(dim=1, keepdim=True)
        qout = n5.query(qo, qw)
        sec = _time(torch, lambda: n5.query(qo, qw, out=qout), 3)
        f5 = 2.0 * ((6 + 6 * F5) * W5 + (L5 - 1) * W5 * W5 + 2 * W5)
        peak = peaks["bf16_tflops_sustained"]
        rows["query_w512"] = {"workload": "2^22 queries, 102 -> 512 x 8 -> 2, BF16, no normals",
                              "queries_per_s": nq / sec,
                              "roofline": {"bound": "tensor", "achieved": f5 * nq / sec / 1e12, "peak": peak,
                                           "unit": "TFLOP/s", "frac": f5 * nq / sec / 1e12 / peak}}
        if only is None:
            cam5 = default_camera(1920, 1080, seed=1)
            img5 = torch.empty(1080, 1920, device="cuda")
            sec = _time(torch, lambda: n5.render(cam5, 8, 8, img5), 1)
            rows["large_render_wave"] = {"workload": "1920 x 1080 x 8 spp (one wave of 16.6M paths), <= 8 bounces, "
                                                     "102 -> 512 x 8 -> 2 BF16 (the full 256-spp render is 32 such "
                                                     "waves)",
                                         "samples_per_s": 1920 * 1080 * 8 / sec, "ms": sec * 1e3,
                                         "queries_per_bounce": n5.render_stats(8)}
    return rows


def query_error(P, net, blob, w, n=65536):
    """Errors of the GPU query against the FP64 oracle on 65,536 rays in the unit ball: max / p99
    |d dist|, hit-decision mismatch rate where |logit| >= 1e-4, and the angle between the GPU and
    oracle Eq. 3 normals on rows both call hits (median / p99 degrees)."""
    import numpy as np
    import torch
    from oracle import mlp as omlp
    rng = np.random.default_rng(13)
    o = rng.normal(size=(n, 3))
    o = (o / np.linalg.norm(o, axis=1, keepdims=True) * rng.uniform(0.1, 1.0, (n, 1))).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    out = net.query(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), normals=True)
    torch.cuda.synchronize()
    ref = omlp.query(omlp.unpack(blob, w["in_freqs"], w["hidden"], w["layers"]), o, d, w["in_freqs"])
    err = np.abs(out["dist"].cpu().numpy() - ref["dist"])
    hit = out["hit"].cpu().numpy().astype(bool)
    clear = np.abs(ref["logit"]) >= 1e-4
    mism = np.mean(hit[clear] != ref["hit"][clear])
    both = hit & ref["hit"]
    cos = np.clip(np.sum(out["normal"].cpu().numpy()[both] * ref["normal"][both], 1), -1, 1)
    ang = np.degrees(np.arccos(cos)) if both.any() else np.zeros(1)
    return {"rays": n, "max_abs_dist": float(err.max()), "p99_abs_dist": float(np.percentile(err, 99)),
            "hit_mismatch_rate": float(mism), "normal_rows": int(both.sum()),
            "normal_angle_deg_median": float(np.median(ang)), "normal_angle_deg_p99": float(np.percentile(ang, 99))}


if __name__ == "__main__":
    sys.exit(main())
