#!/usr/bin/env python3
"""Benchmark: vector fields/s and latency of the dense pyramidal Lucas-Kanade flow at
1024^2 (12-bit particle images, Lamb-Oseen vortex + shear layer, 3 levels, window radius
4, 5 iterations per level), FP16-storage batched form vs plain FP32 single pair, with
the fraction of the HBM roofline.

One step = the whole method (pyramids + all iterations on all levels) for a batch of
pairs through of_compute_batch: one CUDA graph replay of the phase launches (or of the
persistent launch, if the autotuner picks it); inputs are resident in HBM when the
timed region starts and the step's working set is far above the L2 size.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]

Multi-GPU (torchrun, one process per GPU): fields are independent, so each rank runs
its own replica of the batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vector fields/s & p99 latency at 1024², FP16-storage vs FP32, % HBM roofline"
UNIT = "fields/s"
H = W = 1024
LEVELS, RADIUS, ITERS, BITS = 3, 4, 5, 12
WORKLOAD = "pair1024_u16_vortex_shear"
DISTINCT = 8          # distinct seeded pairs; the batch cycles through them


def level_sizes(H, W, L):
    out = []
    for _ in range(L):
        out.append((H, W))
        H, W = (H + 1) // 2, (W + 1) // 2
    return out


def algorithmic_bytes(H, W, L, n, s, raw):
    """Minimum HBM bytes of one field for this dataflow (each byte read or written once):
    pyramids: read raw (raw B/px) once, write every level at s B/px, read levels 1..L-2
    once to build the next; iterations: read I1 and I2 (s each) and the current (u, v)
    (8 B), write the new (u, v) (8 B) per pixel, except that the first iteration on the
    coarsest level reads no flow and the first on a finer level reads the coarse one."""
    lv = level_sizes(H, W, L)
    N = [h * w for h, w in lv]
    pyr = 2 * (raw * N[0] + s * sum(N) + s * sum(N[1:L - 1]))
    it = 0
    for l in range(L):
        for k in range(n):
            rd_flow = 0 if (k == 0 and l == L - 1) else (8 * N[l + 1] if k == 0 else 8 * N[l])
            it += 2 * s * N[l] + rd_flow + 8 * N[l]
    return pyr + it, pyr, it


def unfused_dataflow_bytes(H, W, L, n, s, raw):
    """The same count for the plain dataflow without this implementation's two savings:
    the first reduction re-reads level 0 instead of taking it from the raw read, and every
    iteration reads a full-level estimate (none is skipped at the very first, none comes
    from the coarser level): pyramids read raw, write every level and read levels
    0..L-2 once; iterations read I1, I2 (s each) and the estimate (8 B) and write (8 B)."""
    N = [h * w for h, w in level_sizes(H, W, L)]
    return 2 * (raw * N[0] + s * sum(N) + s * sum(N[:L - 1])) + n * sum(N) * (2 * s + 16)


def algorithmic_bytes_i1grad(H, W, L, n, s, raw):
    """The same for the first-image-gradient variant: per level the window matrices are
    written once (16 B/px, after reading I1 at s B/px) and read by every iteration."""
    tot, pyr, it = algorithmic_bytes(H, W, L, n, s, raw)
    extra = sum(h * w * (s + 16 + 16 * n) for h, w in level_sizes(H, W, L))
    return tot + extra, pyr, it + extra


def pixel_iterations(H, W, L, n):
    return n * sum(h * w for h, w in level_sizes(H, W, L))


# Sources that take no part in the timed step (the serving loop, the allocation-free
# entry point, the host-buffer pipeline): left out of the hash, so that the recorded
# traffic stays attached to the code that produced it.
NOT_IN_STEP = {"server.cu", "noalloc.cu", "host_pipe.cu"}


def kernel_source_hash():
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1306_2461_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")) and f not in NOT_IN_STEP:
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel_hash, variant=False, key="bytes_per_step_full_batch"):
    """DRAM bytes per step (all kernels of one graph replay; or another recorded `key`) from
    the committed ncu summary, if it was taken on this exact kernel source (else None)."""
    name = "batch_step_i1grad_pair1024_traffic.txt" if variant else "batch_step_pair1024_traffic.txt"
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        parts = line.split()
        if len(parts) >= 2 and not line.startswith("#"):
            kv[parts[0]] = parts[1]
    if kv.get("kernel_source_sha1") != kernel_hash:
        return None
    try:
        return float(kv[key])
    except (KeyError, ValueError):
        return None


def dominant_kernel_leg(torch, of, I1, I2, stream, peak, khash, pairs=32, reps=20):
    """The level-0 same-level iteration (the step's dominant kernel) timed live: one-level
    plans run one zero-start iteration, then same-level ones, each a phase launch over the
    batch; 6 and 2 iterations differ by 4 same-level launches that write the interleaved
    estimate, as the level-0 iterations of the step do (the step's sequences are 32 pairs
    each). CUDA events around `reps` graph replays of each on the launching stream."""
    n = min(pairs, len(I1))
    ms = {}
    for iters in (2, 6):
        plan = of.Plan.make(H, W, 1, RADIUS, iters, bits=BITS, storage="f16")
        flows = [of.Flow(plan) for _ in range(n)]
        us = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(n)]
        vs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(n)]
        with torch.cuda.stream(stream):
            for _ in range(3):
                of.compute_batch(flows, I1[:n], I2[:n], us, vs, stream=stream)
            stream.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                of.compute_batch(flows, I1[:n], I2[:n], us, vs, stream=stream)
            b.record(stream)
            stream.synchronize()
        ms[iters] = a.elapsed_time(b) / reps
        for f in flows:
            f.close()
    launch_ms = (ms[6] - ms[2]) / 4
    alg = n * H * W * (2 * 2 + 8 + 8)
    achieved = alg / (launch_ms / 1000.0) / 1e9
    traffic = recorded_traffic(khash, key="dominant_kernel_bytes_per_launch") if n == 32 else None
    return {"kernel": "phase_iter_kernel<uint16_t, 4, SAME, 24> (level-0 same-level iteration)",
            "pairs_per_launch": n, "launch_us": launch_ms * 1000.0, "algorithmic_bytes_per_launch": alg,
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "method": "one-level batches of 6 and 2 iterations timed with CUDA events on the launching stream; "
                      "their difference is 4 same-level launches"}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, pw, mx, reasons = [], [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except (ValueError, IndexError):
                continue
            try:
                pw.append(float(f[3]))
            except (ValueError, IndexError):
                pass
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "power_w": statistics.median(pw) if pw else None, "samples": len(sm)}


def aggregate(local_ms, local_fields, world):
    """Replicas (fields are independent): every rank timed its own batch; the job's time
    is the slowest rank's and its fields are all ranks' together. Returns (ms, fields)."""
    if world <= 1:
        return float(local_ms), float(local_fields)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    f = torch.tensor([float(local_fields)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return float(t.item()), float(f.item())


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, np.float64), q)) if xs else None


# ------------------------------------------------------------------ reference arm
def cpu_oracle_sample(budget_s=12.0, max_pairs=8, workloads=True):
    """The CPU baseline: the FP64 oracle, as it stands, on whole 1024^2 pairs of the
    workload: as many as fit in about budget_s seconds (at least one) on all host cores,
    and one pair on one core. Also the oracle's fields the GPU fields are compared with:
    the first pair (and the same pair on its FP16-rounded pyramid) and, with `workloads`,
    one pair of the 2048^2 workload and the smallest pair of the mixed batch (those inputs
    are rendered here and reused by the GPU legs)."""
    import oracle
    from paper_1306_2461_gb300 import synth
    oracle.build()
    pairs = [synth.make_c2(H, W, seed=1 + 7919 * i) for i in range(2)]
    t0 = time.perf_counter()
    done = 0
    first = None
    while done < max_pairs:
        p = pairs[done % len(pairs)]
        uv = oracle.flow(p.I1, p.I2, LEVELS, RADIUS, ITERS)
        if first is None:
            first = uv
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    nt = oracle.threads()
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.flow(pairs[0].I1, pairs[0].I2, LEVELS, RADIUS, ITERS)
    single = time.perf_counter() - t1
    oracle.set_threads(nt)
    res = {"value": done / dt, "pairs": done, "secs": dt, "threads": nt, "first": first, "single_s": single,
           "first_stored_f16": oracle.flow_stored(pairs[0].I1, pairs[0].I2, LEVELS, RADIUS, ITERS, "f16")}
    if workloads:
        c3 = synth.make_c3()
        res["c3"] = (c3, oracle.flow(c3.I1, c3.I2, 4, 3, 6))
        distinct = synth.make_batch(16, seed=3)
        small = min(range(16), key=lambda i: distinct[i].I1.size)
        res["c4"] = (distinct, small, oracle.flow(distinct[small].I1, distinct[small].I2, 3, 4, 5))
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from paper_1306_2461_gb300 import synth
    oracle.build()
    p = synth.make_c2(H, W, seed=1)
    for _ in range(args.warmup):
        oracle.flow(p.I1, p.I2, LEVELS, RADIUS, ITERS)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.flow(p.I1, p.I2, LEVELS, RADIUS, ITERS)
        t.append(time.perf_counter() - t0)
    total = sum(t)
    val = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "H": H, "W": W, "levels": LEVELS,
                                            "radius": RADIUS, "iterations": ITERS, "pairs_per_step": 1},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"one whole {H}x{W} pair per step, FP64 C oracle with OpenMP"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------ our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the single-pair and e2e legs")
    ap.add_argument("--no-autotune", action="store_true", help="run the batched launch with the default tuning")
    ap.add_argument("--tile-h", type=int, default=0,
                    help="with --no-autotune: the iteration tile height of the forced tuning (0: the default)")
    ap.add_argument("--stage", type=int, default=1,
                    help="with --no-autotune: 1 (default) stages each tile's estimate and I2 window in shared "
                         "memory with TMA copies, 0 gathers them from global memory")
    ap.add_argument("--branches", type=int, default=0,
                    help="with --no-autotune: the default tuning in this many concurrent launch sequences")
    ap.add_argument("--i1grad", action="store_true",
                    help="time the first-image-gradient variant (window matrix fixed per level) as the step")
    ap.add_argument("--table1", action="store_true",
                    help="sweep levels {3,4} x iterations 1..7 at 1792x384, r = 10 (synthetic Table 1) and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    # the CPU oracle runs before the first GPU call (no fork after CUDA init)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(workloads=not args.no_extras and not args.i1grad)

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1306_2461_gb300 import build as libbuild
    libbuild.build()
    from paper_1306_2461_gb300 import of, synth
    if args.table1:
        if rank == 0:
            print(json.dumps(table1_sweep(torch, of, synth)), flush=True)
        return 0

    B = args.batch
    src = [synth.make_c2(H, W, seed=1 + 7919 * (i + rank * DISTINCT)) for i in range(DISTINCT)]
    dev = lambda a: torch.from_numpy(a.astype(np.int32)).cuda().to(torch.uint16)
    I1 = [dev(src[i % DISTINCT].I1) for i in range(B)]
    I2 = [dev(src[i % DISTINCT].I2) for i in range(B)]
    stream = torch.cuda.Stream()
    plan16 = of.Plan.make(H, W, LEVELS, RADIUS, ITERS, bits=BITS, storage="f16",
                          flags=of.OF_FLAG_I1GRAD if args.i1grad else 0)
    flows = [of.Flow(plan16) for _ in range(B)]
    us = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(B)]
    vs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in range(B)]

    def step():
        of.compute_batch(flows, I1, I2, us, vs, stream=stream)

    # the library's autotuner picks how the batched launch runs (outside the timed region)
    tuning = None
    if not args.no_autotune:
        from paper_1306_2461_gb300 import autotune
        tuning = autotune.tune(flows, I1, I2, us, vs, stream=stream, reps=2, save=False)
    elif args.branches > 1 or args.tile_h or not args.stage:
        of.tuning_set(flows[0].plan, of.batch_size_class(flows), branches=max(args.branches, 0),
                      tile_h=args.tile_h, stage_i2=args.stage)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    for f in flows:
        if f.sync_status() != of.OF_OK:
            raise RuntimeError("device status not OK after warm-up")

    # timed region: K steps, events around every launch on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_host0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        t_host = time.perf_counter() - t_host0
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, fields = aggregate(ev[0][0].elapsed_time(ev[-1][1]), B * args.steps, world)
    value = fields / (total_ms / 1000.0)

    extras = {}
    if not args.no_extras and not args.i1grad:
        extras = extra_legs(args, torch, of, synth, src, I1, I2, us, vs, stream, plan16, flows, world, cpu)

    # accuracy of the timed configuration on one pair (outside the timed region)
    p0 = src[0]
    u0 = us[0].cpu().double().numpy()
    v0 = vs[0].cpu().double().numpy()
    m = (RADIUS + 2) * 2 ** (LEVELS - 1)
    e = np.sqrt((u0 - p0.u_gt) ** 2 + (v0 - p0.v_gt) ** 2)[m:-m, m:-m]
    for f in flows:
        if f.sync_status() != of.OF_OK:
            raise RuntimeError("device status not OK after the timed region")

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    alg, alg_pyr, alg_it = (algorithmic_bytes_i1grad if args.i1grad else algorithmic_bytes)(H, W, LEVELS, ITERS, 2, 2)
    phased = tuning["best"]["phased"] if tuning else 1
    branches = (tuning["best"]["branches"] if tuning else max(args.branches, 1)) if phased else 1
    # the batch runs as `branches` concurrent sequences over runs of equal-size pairs (run k
    # ends at the first pair count >= B k / branches), each in launches of at most 64 pairs
    nb = min(branches, B)
    cuts = [0] + [-(-B * k // nb) for k in range(1, nb)] + [B]
    groups = sum((cuts[k + 1] - cuts[k] + 63) // 64 for k in range(nb))
    if args.i1grad:
        launches_per_step = groups * (max(LEVELS - 1, 1) + LEVELS + LEVELS * ITERS)
        step_kernels = (f"batch step: {groups * max(LEVELS - 1, 1)} phase_pyr_kernel + {groups * LEVELS} "
                        f"phase_hess_kernel + {groups * LEVELS * ITERS} phase_i1_iter_kernel launches")
    else:
        launches_per_step = groups * (max(LEVELS - 1, 1) + LEVELS * ITERS) if phased else 1
        step_kernels = (f"batch step: {groups * max(LEVELS - 1, 1)} phase_pyr_kernel + {groups * LEVELS * ITERS} "
                        "phase_iter_kernel launches" if phased else "batch step: 1 persistent batch_kernel launch")
    peak, peak_kind = measured_peaks()
    launch_ms = statistics.mean(step_ms)
    achieved = alg * B / (launch_ms / 1000.0) / 1e9
    khash = kernel_source_hash()
    traffic = recorded_traffic(khash, args.i1grad)
    clocks = clk.summary()
    # the dominant kernel alone, timed live (after the timed region, rank 0)
    dominant = None if args.i1grad else dominant_kernel_leg(torch, of, I1, I2, stream, peak, khash)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": "f16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "bits": BITS, "levels": LEVELS, "radius": RADIUS,
                   "iterations": ITERS, "pairs_per_step": B, "distinct_pairs": DISTINCT,
                   "form": "batched (of_compute_batch), one CUDA graph replay per step",
                   "method": ("first-image-gradient variant (window matrix fixed per level)" if args.i1grad
                              else "second-image gradient at the displaced position"),
                   "tuning": ({k: tuning["best"][k] for k in ("generic_sums", "stage_i2", "blocks_per_sm", "phased",
                                                               "prefetch", "tile_h", "branches", "fusion", "strip")}
                              if tuning else ("default (autotuner off)"
                                              if args.branches <= 1 and not args.tile_h and args.stage else
                                              f"forced (autotuner off): tile_h {args.tile_h or 'default'}, stage "
                                              f"{args.stage}, {max(args.branches, 1)} concurrent sequences")),
                   "l2": "no flush: per-step working set ~%.1f GB >> 129 MB L2" % (
                       B * (of.workspace_bytes(plan16) + 4 * H * W) / 1e9),
                   "parallelism": f"replicas x{world}"},
        "autotune_candidates_ms": ([[c["generic_sums"], c["stage_i2"], c["blocks_per_sm"], c["phased"], c["prefetch"],
                                     c["tile_h"], c["branches"], c["fusion"], c["strip"], round(c["ms"], 3)]
                                    for c in tuning["candidates"]] if tuning else None),
        "autotune_candidate_columns": ["generic_sums", "stage_i2", "blocks_per_sm", "phased", "prefetch", "tile_h",
                                       "branches", "fusion", "strip", "ms"],
        "latency_ms": {"step_p50": percentile(step_ms, 50), "step_p99": percentile(step_ms, 99),
                       "step_max": max(step_ms)},
        "mpix_iter_per_s": pixel_iterations(H, W, LEVELS, ITERS) * value / 1e6,
        "epe_vs_ground_truth_px": {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max()),
                                   "margin_px": m},
        "roofline": {"bound": "hbm", "kernel": step_kernels,
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": traffic,
                     "timed_unit": "one step = one CUDA graph launch, CUDA events around each on the launching stream",
                     "algorithmic_bytes_per_step": alg * B,
                     "algorithmic_bytes_per_field": {"total": alg, "pyramids": alg_pyr, "iterations": alg_it},
                     "unfused_dataflow": None if args.i1grad else {
                         "bytes_per_field": unfused_dataflow_bytes(H, W, LEVELS, ITERS, 2, 2),
                         "frac": unfused_dataflow_bytes(H, W, LEVELS, ITERS, 2, 2) * B / (launch_ms / 1000.0) / 1e9 / peak,
                         "note": "the same time against the byte count of a dataflow that re-reads level 0 for the "
                                 "first reduction and reads a full-level estimate at every iteration"},
                     "dominant_kernel": dominant,
                     "kernel_source_sha1": khash},
        "gpu_launches": args.steps * launches_per_step,
        "host_wall_s": t_host,
    }
    if clocks:
        line["clocks"] = clocks
    line.update(extras)
    if cpu is not None:
        uo, vo = cpu["first"]
        us16, vs16 = cpu["first_stored_f16"]
        line["cpu_baseline"] = {"value": cpu["value"], "unit": UNIT, "cores": cpu["threads"], "kind": "oracle",
                                "sample": f"{cpu['pairs']} whole {H}x{W} pairs of the workload in {cpu['secs']:.1f} s "
                                          "(FP64 C oracle, OpenMP)",
                                "single_thread": {"value": 1.0 / cpu["single_s"], "unit": UNIT, "cores": 1,
                                                  "sample": f"one whole {H}x{W} pair in {cpu['single_s']:.1f} s"},
                                "cpu_model": cpu_model()}
        # the timed configuration's field of the first pair against the oracle's: over every
        # interior pixel; over those whose FP64 result the FP16 rounding of the pyramid
        # itself moves by less than half the tolerance (the others counted); and against
        # the oracle run on the FP16-rounded pyramid (the implementation check)
        d = np.maximum(np.abs(u0 - uo), np.abs(v0 - vo))[m:-m, m:-m]
        sens = (np.maximum(np.abs(us16 - uo), np.abs(vs16 - vo)) > 0.5 * 2e-2)[m:-m, m:-m]
        dimpl = np.maximum(np.abs(u0 - us16), np.abs(v0 - vs16))[m:-m, m:-m]
        line["vs_oracle_px"] = {"max": float(d.max()), "rms": float(np.sqrt((d ** 2).mean())),
                                "p99_9": float(np.percentile(d, 99.9)), "margin_px": m,
                                "max_rounding_aware": float(d[~sens].max()), "storage_sensitive_px": int(sens.sum()),
                                "compared_px": int(d.size),
                                "max_vs_oracle_on_fp16_pyramid": float(dimpl.max()),
                                "note": "FP16-storage batched field vs the FP64 oracle, interior pixels. max: every "
                                        "pixel; max_rounding_aware: pixels whose FP64 result the FP16 rounding of the "
                                        "pyramid moves by < 1e-2 px (the storage-sensitive ones counted); "
                                        "max_vs_oracle_on_fp16_pyramid: against the oracle run on the rounded pyramid. "
                                        "Stated tolerance 2e-2 max, 5e-3 RMS"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def extra_legs(args, torch, of, synth, src, I1, I2, us, vs, stream, plan16, flows, world=1, cpu=None):
    """Outside the headline timed region: the plain FP32 single-pair form (the comparison
    the target names), the first-image-gradient variant, the batch at FP32 storage, e2e
    through the C ABI with host buffers (whole job over all ranks, like the headline),
    and the serving loop. The single-pair, variant, FP32-batch and serving legs are this
    rank's GPU alone."""
    out = {}
    K = max(args.steps, 20)
    # plain FP32 single pair, one of_compute (graph replay) per field; the same at FP16
    # storage, and the first-image-gradient variant (window matrix fixed per level)
    for key, storage, flags in (("single_pair_f32", "f32", 0), ("single_pair_f16", "f16", 0),
                                ("single_pair_f16_i1grad", "f16", of.OF_FLAG_I1GRAD)):
        plan = of.Plan.make(H, W, LEVELS, RADIUS, ITERS, bits=BITS, storage=storage, flags=flags)
        with of.Flow(plan) as f, torch.cuda.stream(stream):
            for _ in range(5):
                f.compute(I1[0], I2[0], us[0], vs[0], stream=stream)
            stream.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            for k in range(K):
                evs[k][0].record(stream)
                f.compute(I1[k % 4], I2[k % 4], us[0], vs[0], stream=stream)   # 4 = graph cache size
                evs[k][1].record(stream)
            stream.synchronize()
            lat = [a.elapsed_time(b) for a, b in evs]
            tot = evs[0][0].elapsed_time(evs[-1][1])
            # accuracy of this form on the first pair (outside the timed region)
            f.compute(I1[0], I2[0], us[0], vs[0], stream=stream)
            stream.synchronize()
        m = (RADIUS + 2) * 2 ** (LEVELS - 1)
        e = np.sqrt((us[0].cpu().double().numpy() - src[0].u_gt) ** 2 +
                    (vs[0].cpu().double().numpy() - src[0].v_gt) ** 2)[m:-m, m:-m]
        out[key] = {"fields_per_s": K / (tot / 1000.0), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                    "epe_vs_ground_truth_px": {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max())}}
    # the first-image-gradient variant in the batched form (phase launches), same workload
    plan_v = of.Plan.make(H, W, LEVELS, RADIUS, ITERS, bits=BITS, storage="f16", flags=of.OF_FLAG_I1GRAD)
    fv = [of.Flow(plan_v) for _ in range(len(flows))]
    with torch.cuda.stream(stream):
        for _ in range(3):
            of.compute_batch(fv, I1, I2, us, vs, stream=stream)
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        Kv = max(5, args.steps // 2)
        a.record(stream)
        for _ in range(Kv):
            of.compute_batch(fv, I1, I2, us, vs, stream=stream)
        b.record(stream)
        stream.synchronize()
    m = (RADIUS + 2) * 2 ** (LEVELS - 1)
    e = np.sqrt((us[0].cpu().double().numpy() - src[0].u_gt) ** 2 +
                (vs[0].cpu().double().numpy() - src[0].v_gt) ** 2)[m:-m, m:-m]
    out["batched_f16_i1grad"] = {"fields_per_s": len(fv) * Kv / (a.elapsed_time(b) / 1000.0),
                                 "ms_per_step": a.elapsed_time(b) / Kv,
                                 "epe_vs_ground_truth_px": {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max())}}
    for f in fv:
        f.close()
    # the same batch at FP32 storage of the reduced levels (autotuned like the headline)
    plan32 = of.Plan.make(H, W, LEVELS, RADIUS, ITERS, bits=BITS, storage="f32")
    f32 = [of.Flow(plan32) for _ in range(len(flows))]
    t32 = None
    if not args.no_autotune:
        from paper_1306_2461_gb300 import autotune
        t32 = autotune.tune(f32, I1, I2, us, vs, stream=stream, reps=2, save=False)["best"]
    with torch.cuda.stream(stream):
        for _ in range(3):
            of.compute_batch(f32, I1, I2, us, vs, stream=stream)
        stream.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        K32 = max(5, args.steps // 2)
        a.record(stream)
        for _ in range(K32):
            of.compute_batch(f32, I1, I2, us, vs, stream=stream)
        b.record(stream)
        stream.synchronize()
    e = np.sqrt((us[0].cpu().double().numpy() - src[0].u_gt) ** 2 +
                (vs[0].cpu().double().numpy() - src[0].v_gt) ** 2)[m:-m, m:-m]
    out["batched_f32"] = {"fields_per_s": len(f32) * K32 / (a.elapsed_time(b) / 1000.0),
                          "ms_per_step": a.elapsed_time(b) / K32,
                          "tuning": ({k: t32[k] for k in ("generic_sums", "stage_i2", "blocks_per_sm", "phased",
                                                          "prefetch", "tile_h", "branches", "fusion", "strip")} if t32 else None),
                          "epe_vs_ground_truth_px": {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max())}}
    for f in f32:
        f.close()
    # e2e: host (pinned) frames in, device compute, host flow fields out, every step
    B = len(flows)
    h1 = [torch.from_numpy(src[i % len(src)].I1.astype(np.int32)).to(torch.uint16).pin_memory() for i in range(B)]
    h2 = [torch.from_numpy(src[i % len(src)].I2.astype(np.int32)).to(torch.uint16).pin_memory() for i in range(B)]
    hu = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(B)]
    hv = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(B)]

    def e2e_serial():
        for i in range(B):
            I1[i].copy_(h1[i], non_blocking=True)
            I2[i].copy_(h2[i], non_blocking=True)
        of.compute_batch(flows, I1, I2, us, vs, stream=stream)
        for i in range(B):
            hu[i].copy_(us[i], non_blocking=True)
            hv[i].copy_(vs[i], non_blocking=True)

    def e2e_pipelined():
        of.compute_batch_host(flows, h1, h2, hu, hv, I1, I2, us, vs, stream=stream, chunk=0)

    Ke = max(3, args.steps // 2)
    for key, fn, path in (("e2e", e2e_pipelined, "pinned host frames -> of_compute_batch_host (default chunks of about 8 Mpx, a quarter and a half of that at either end, "
                                                 "alternating between two compute streams; uploads and "
                                                 "downloads on two copy streams overlap the launches) -> pinned host u, v"),
                          ("e2e_unpipelined", e2e_serial, "pinned host frames -> of_compute_batch -> pinned host u, v, "
                                                          "copies and launch in order on one stream")):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            stream.synchronize()
            if world > 1:
                torch.distributed.barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(Ke):
                fn()
            b.record(stream)
            stream.synchronize()
        ms, fields = aggregate(a.elapsed_time(b), B * Ke, world)
        out[key] = {"value": fields / (ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": world * B * 2 * H * W * 2,
                    "d2h_bytes_per_step": world * B * 2 * H * W * 4, "steps": Ke, "path": path}
    out["serving"], out["serving_sweep"] = serving_leg(torch, synth)
    out.update(workload_legs(torch, of, synth, stream, cpu))
    out["table1_synthetic"] = table1_sweep(torch, of, synth, batch=16, reps=10)["table1_synthetic"]
    return out


def _epe(u, v, p, m):
    e = np.sqrt((u - p.u_gt) ** 2 + (v - p.v_gt) ** 2)[m:-m, m:-m]
    return {"rms": float(np.sqrt((e ** 2).mean())), "max": float(e.max())}


def workload_legs(torch, of, synth, stream, cpu=None, steps=10):
    """The other workloads, batched and timed like the headline (graph replays, CUDA events),
    each with its end-point error against the analytic field and its distance from the FP64
    oracle on one pair:
      c3: 2048^2 12-bit with a low-seeding band, band-limited flow up to 10 px; 4 levels, r = 3,
          6 iterations, FP16 storage with FP64 solves on ill-conditioned pixels; 8 pairs per step
          (one rendered pair, repeated);
      c4: 64 pairs of mixed sizes (256^2, 512^2, 1024^2, 2048 x 1024 uint8, uniform + vortex flow);
          3 levels, r = 4, 5 iterations, FP16 storage; 16 rendered pairs, cycled."""
    from paper_1306_2461_gb300 import autotune
    out = {}

    def timed(flows, I1, I2, us, vs):
        autotune.tune(flows, I1, I2, us, vs, stream=stream, reps=2, save=False)
        with torch.cuda.stream(stream):
            for _ in range(3):
                of.compute_batch(flows, I1, I2, us, vs, stream=stream)
            stream.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                of.compute_batch(flows, I1, I2, us, vs, stream=stream)
            b.record(stream)
            stream.synchronize()
        return a.elapsed_time(b) / steps

    dev16 = lambda a: torch.from_numpy(a.astype(np.int32)).cuda().to(torch.uint16)
    # c3
    have = cpu is not None and "c3" in cpu
    p, (uo, vo) = cpu["c3"] if have else (synth.make_c3(), (None, None))
    L3, r3, n3 = 4, 3, 6
    plan = of.Plan.make(2048, 2048, L3, r3, n3, bits=12, storage="f16", fp64_cond=1e3)
    B3 = 8
    flows = [of.Flow(plan) for _ in range(B3)]
    I1 = [dev16(p.I1)] * B3
    I2 = [dev16(p.I2)] * B3
    us = [torch.empty((2048, 2048), device="cuda") for _ in range(B3)]
    vs = [torch.empty((2048, 2048), device="cuda") for _ in range(B3)]
    ms = timed(flows, I1, I2, us, vs)
    u = us[0].cpu().double().numpy()
    v = vs[0].cpu().double().numpy()
    m = (r3 + 2) * 2 ** (L3 - 1)
    with of.Flow(plan) as f1:   # the batched field equals one of_compute of the pair
        u1, v1 = f1.compute(I1[0], I2[0])
        torch.cuda.synchronize()
        same = bool(torch.equal(u1, us[0]) and torch.equal(v1, vs[0]))
    leg = {"fields_per_s": B3 / (ms / 1000.0), "ms_per_step": ms, "pairs_per_step": B3,
           "batched_equals_single_pair": same,
           "mpix_iter_per_s": pixel_iterations(2048, 2048, L3, n3) * B3 / ms / 1000.0,
           "epe_vs_ground_truth_px": _epe(u, v, p, m)}
    if have:
        reach = sum((r3 + 1) * n3 * 2 ** l for l in range(L3))
        rows = np.arange(2048)
        outside = (rows < 0.4 * 2048 - reach) | (rows >= 0.6 * 2048 + reach)
        d = np.maximum(np.abs(u - uo), np.abs(v - vo))
        dm, do = d[m:-m, m:-m], d[outside][:, m:-m]
        leg["vs_oracle_px"] = {"max": float(dm.max()), "rms": float(np.sqrt((dm ** 2).mean())),
                               "max_outside_band": float(do.max()), "rms_outside_band": float(np.sqrt((do ** 2).mean())),
                               "p99_9_outside_band": float(np.percentile(do, 99.9)),
                               "within_2e-2_outside_band": float((do <= 2e-2).mean()),
                               "note": f"FP16 storage vs the unrounded FP64 oracle over every interior pixel (no "
                                       f"exclusion of near-singular or unstable windows, which the parity tests count "
                                       f"and leave out); the low-seeding band widened by {reach} px is where the "
                                       f"method is chaotic"}
    out["c3_2048_lowseed_f16_fp64"] = leg
    for f in flows:
        f.close()
    del I1, I2, us, vs
    # c4
    have = cpu is not None and "c4" in cpu
    if have:
        distinct, small, (uo, vo) = cpu["c4"]
    else:
        distinct = synth.make_batch(16, seed=3)
        small = min(range(16), key=lambda i: distinct[i].I1.size)
    B4 = 64
    pairs = [distinct[i % 16] for i in range(B4)]
    plans = [of.Plan.make(*q.shape, 3, 4, 5, bits=8, storage="f16") for q in pairs]
    flows = [of.Flow(pl) for pl in plans]
    I1 = [torch.from_numpy(q.I1).cuda() for q in pairs]
    I2 = [torch.from_numpy(q.I2).cuda() for q in pairs]
    us = [torch.empty(q.shape, device="cuda") for q in pairs]
    vs = [torch.empty(q.shape, device="cuda") for q in pairs]
    ms = timed(flows, I1, I2, us, vs)
    m = (4 + 2) * 4
    epes = [_epe(us[i].cpu().double().numpy(), vs[i].cpu().double().numpy(), pairs[i], m)["rms"] for i in range(16)]
    px = sum(q.I1.size for q in pairs)
    leg = {"fields_per_s": B4 / (ms / 1000.0), "ms_per_step": ms, "pairs_per_step": B4,
           "mpix_per_step": px / 1e6,
           "epe_vs_ground_truth_px": {"rms_mean_over_pairs": float(np.mean(epes)), "rms_max_over_pairs": float(max(epes))}}
    if have:
        d = np.maximum(np.abs(us[small].cpu().double().numpy() - uo),
                       np.abs(vs[small].cpu().double().numpy() - vo))[m:-m, m:-m]
        leg["vs_oracle_px"] = {"pair_shape": list(pairs[small].I1.shape), "max": float(d.max()),
                               "rms": float(np.sqrt((d ** 2).mean()))}
    out["c4_mixed64_u8_f16"] = leg
    for f in flows:
        f.close()
    return out


def table1_sweep(torch, of, synth, batch=16, reps=20):
    """Synthetic analogue of Table 1: for levels in {3, 4} and iterations 1..7 at the
    paper's region of interest (1792 x 384, 8-bit, r = 10), the error of the field
    relative to the 7-iteration field of the same level count (RMS of the difference over
    RMS of that field, in %), and fields/s of the plain FP32 single pair and of the
    FP16 batched launch (batch pairs per launch)."""
    Hr, Wr, r = 384, 1792, 10
    p = synth.make_bfs(Hr, Wr, seed=5)
    I1 = torch.from_numpy(p.I1).cuda()
    I2 = torch.from_numpy(p.I2).cuda()
    s = torch.cuda.Stream()
    rows = []
    m = (r + 2) * 4
    for L in (3, 4):
        fields = {}
        for n in range(1, 8):
            plan = of.Plan.make(Hr, Wr, L, r, n, bits=8, storage="f32")
            with of.Flow(plan) as f, torch.cuda.stream(s):
                for _ in range(3):
                    u, v = f.compute(I1, I2, stream=s)
                s.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                for _ in range(reps):
                    f.compute(I1, I2, u, v, stream=s)
                b.record(s)
                s.synchronize()
                single = reps / (a.elapsed_time(b) / 1000.0)
                fields[n] = (u.cpu().double().numpy(), v.cpu().double().numpy())
            plan16 = of.Plan.make(Hr, Wr, L, r, n, bits=8, storage="f16")
            flows = [of.Flow(plan16) for _ in range(batch)]
            with torch.cuda.stream(s):
                for _ in range(3):
                    of.compute_batch(flows, [I1] * batch, [I2] * batch, stream=s)
                s.synchronize()
                a.record(s)
                for _ in range(max(3, reps // 4)):
                    of.compute_batch(flows, [I1] * batch, [I2] * batch, stream=s)
                b.record(s)
                s.synchronize()
            batched = batch * max(3, reps // 4) / (a.elapsed_time(b) / 1000.0)
            for f in flows:
                f.close()
            rows.append({"levels": L, "iterations": n, "single_f32_fields_per_s": single,
                         "batched_f16_fields_per_s": batched})
        u7, v7 = fields[7]
        ref = np.sqrt(np.mean((u7 ** 2 + v7 ** 2)[m:-m, m:-m]))
        for row in rows[-7:]:
            un, vn = fields[row["iterations"]]
            d = np.sqrt(np.mean(((un - u7) ** 2 + (vn - v7) ** 2)[m:-m, m:-m]))
            row["error_pct_vs_7_iterations"] = 100.0 * d / ref
            e = np.sqrt((un - p.u_gt) ** 2 + (vn - p.v_gt) ** 2)[m:-m, m:-m]
            row["epe_rms_px"] = float(np.sqrt((e ** 2).mean()))
    return {"table1_synthetic": rows, "config": {"workload": "roi1792x384_u8_bfs", "radius": r,
                                                 "batch": batch}}


def serving_leg(torch, synth, rates=(2000.0, 4000.0, 6000.0, 8000.0), frames_per_stream=112, warm_frames=16):
    """16 time-resolved camera streams (8 x 512^2, 6 x 1024^2, 2 x 2048^2, 12-bit; the 4:3:1
    mix), each a sequence of consecutive frames of particles advected by RK4 through a
    drifting vortex street (generated on the device, copied to pinned host memory: no frame
    repeats), served with continuous batching and resident previous-frame pyramids under
    open-loop Poisson arrivals, at each offered load in `rates` (pairs/s over all streams).
    Every stream has exactly frames_per_stream arrivals; fields are counted from the
    warm_frames-th arrival time until the first stream's last arrival. Latency = completion
    seen by the server's worker - scheduled arrival (the host-to-device copy of the frame
    included; no device-to-host copy of the field). EPE: one served pair per stream (frames
    k, k+1 in the middle of the sequence) against the RK4 one-frame displacement."""
    from paper_1306_2461_gb300 import serve, synth_gpu
    n = sum(c for _, _, c in synth.SERVE_MIX)
    kmid = frames_per_stream // 2
    seqs = []
    t_gen = time.perf_counter()
    k = 0
    for H, W, cnt in synth.SERVE_MIX:
        for _ in range(cnt):
            gs = synth_gpu.GpuParticleStream(H, W, seed=4 * 1009 + k)
            frames, gts = synth_gpu.render_sequence(gs, frames_per_stream, gt_at={kmid})
            seqs.append((H, W, frames, gts[kmid]))
            k += 1
    t_gen = time.perf_counter() - t_gen
    m = (RADIUS + 2) * 2 ** (LEVELS - 1)
    sweep = []
    for ri, rate in enumerate(rates):
        per = rate / n
        with serve.Server(levels=LEVELS, radius=RADIUS, iterations=ITERS, bits=BITS, storage="f16",
                          hbm_budget_bytes=64 << 30, max_batch=64, max_inflight=2) as srv:
            streams = [(srv.open_stream(H, W), frames) for H, W, frames, _ in seqs]
            arrivals, last = synth_gpu.per_stream_arrivals(n, frames_per_stream, per, seed=4 + ri)
            warm = warm_frames / per
            end = min(last)
            results, _, kept = serve.run_open_loop(srv, streams, arrivals, warmup_s=warm, end_s=end,
                                                   keep=[(s, kmid + 1) for s in range(n)])
            summ = serve.summarize(results, end - warm)
            st = srv.stats()
        epe = {}
        for s, (H, W, _, (ug, vg)) in enumerate(seqs):
            if (s, kmid + 1) not in kept:
                continue
            u, v = kept[(s, kmid + 1)]
            e = torch.sqrt((u - ug) ** 2 + (v - vg) ** 2)[m:-m, m:-m]
            epe.setdefault(f"{H}x{W}", []).append(float(torch.sqrt((e ** 2).mean())))
        summ.update({"offered_pairs_per_s": rate, "window_s": end - warm, "ticks": st["ticks"],
                     "epe_rms_px": {k2: float(np.mean(v2)) for k2, v2 in epe.items()}})
        sweep.append(summ)
    head = dict(sweep[0])
    head.update({"streams": "8x512^2 + 6x1024^2 + 2x2048^2, 12-bit, time-resolved (no frame repeats)",
                 "frames_per_stream": frames_per_stream, "generation_s": t_gen,
                 "note": "latency from the scheduled arrival; EPE of one served pair per stream vs the RK4 displacement"})
    return head, sweep


if __name__ == "__main__":
    sys.exit(main())
