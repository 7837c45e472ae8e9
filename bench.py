#!/usr/bin/env python3
"""Benchmark of the stochastic Barnes-Hut hot path on one or more GB300s.

A step is one pass of the whole hot path over one batch: the GPU tree build (bounds, Morton
codes, radix sort, topology, aggregates) followed by the stratified path estimator at every query.
The default workload is the winding-number problem: 2^20 oriented, area-weighted surface samples on
a union of 8 random ellipsoids, evaluated on the 256^3 cell-centred grid of their bounding box,
S = 1 path per subdomain, leaf size 1.

Printed (rank 0, one JSON line): whole-job queries/s over the timed steps, the end-to-end number
through the public API with pinned host buffers, the roofline of the estimator kernel, the CPU
oracle's throughput, clocks sampled during the timed region, and the equal-median-error comparison
with the project's own GPU Barnes-Hut (theta sweep, log-log interpolation).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

With N > 1 it runs under torchrun, one replica per GPU (each rank its own seeded problem), no
collective on the data path; the timed region is bracketed by barriers and the time is the maximum
over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "queries/sec at equal median rel. error vs own GPU deterministic BH; % roofline"
L2_BYTES = 129 * 1024 * 1024
L2_NOTE = "L2 flushed before every timed iteration (a 258 MiB device write, outside the timed events)"
_FLUSH = {}


def flush_l2(dev):
    """Write a buffer twice the size of L2 on the current stream, so that the next timed launch
    finds none of its inputs (nor the previous iteration's tree) in L2."""
    import torch
    buf = _FLUSH.get(str(dev))
    if buf is None:
        buf = _FLUSH[str(dev)] = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    buf.fill_(float(len(_FLUSH)))

# FP32 floating-point operations of one kernel term as written in the CUDA kernels (an FMA counts
# 2, a multiply, add, rsqrt or exp 1): Coulomb 3 sub + r^2 with eps^2 (3 FMA) + rsqrt + scale +
# accumulate; winding 3 sub + r^2 (2 FMA + mul) + rsqrt + r^-3 (2 mul) + (p - q).N (2 FMA + mul) +
# mul + accumulate (the 1/(4 pi) is applied once per swap); smooth distance 3 sub + r^2 (2 FMA +
# mul) + r (rsqrt, mul) + compare + alpha (d - ref) (sub, mul) + exp + FMA; affine 3 sub +
# g.(p - q) (2 FMA + mul) + add + mul + add.
FLOPS_PER_TERM = {"coulomb": 12, "winding": 18, "smoothdist": 16, "affine": 11}
# FP32 lanes per SM of a Blackwell SM (two flops per lane per cycle with an FMA); the SM count is
# read from the device and the clock from the samples taken during the timed region
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(sms: int, sm_mhz: float) -> float:
    """Dense FP32 FMA peak: SMs x 128 lanes x 2 flop x clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def peak_clock_mhz(clk):
    """The SM clock the peak is taken at: the maximum SM clock nvidia-smi reported while the timed
    region ran (clocks.max.sm); else the measured one in MEASURED_PEAKS.json; else the
    GB300's nominal maximum. Returns (MHz, where it came from)."""
    if clk and clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"]), "clocks.max.sm sampled during the timed region"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, KeyError, ValueError):
        return 2070.0, "nominal maximum SM clock of a GB300 (no sample)"


def workload_by_name(name: str, rank: int = 0):
    from paper_2506_02219_gb300 import workloads as W
    b = W.BASE_SEED
    if name == "winding":
        return W.winding_ellipsoids(seed=b + 1 + 1000 * rank)
    if name == "winding_random":
        return W.winding_ellipsoids_random(seed=b + 1 + 1000 * rank)
    if name == "cube":
        return W.coulomb_cube(seed=b + 0 + 1000 * rank)
    if name == "slice_coulomb":
        return W.slice_plane_shapes(kernel="coulomb", seed=b + 2 + 1000 * rank)
    if name == "slice_smoothdist":
        return W.slice_plane_shapes(kernel="smoothdist", seed=b + 2 + 1000 * rank)
    if name == "far_coulomb":
        return W.far_field_coulomb(seed=b + 1 + 1000 * rank)
    raise ValueError(name)


# ------------------------------------------------------------------------------------------------
# distributed plumbing (also exercised on CPU with gloo by the tests)
# ------------------------------------------------------------------------------------------------
def dist_env():
    """(rank, world_size, local_rank) from the torchrun environment (defaults: single process)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def weak_scaling_value(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: every rank processed units_per_rank in at most max_seconds."""
    return units_per_rank * world / max_seconds


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not mhz:
            return None
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(mhz)}


# ------------------------------------------------------------------------------------------------
# helpers
# ------------------------------------------------------------------------------------------------
def _kernel_kwargs(wl):
    return dict(kernel=wl.kernel, softening=wl.softening, alpha=wl.alpha)


def rel_error(kind, est, ref):
    """Per-query relative error: |F^ - F| / |F|; winding numbers / max(|F|, 1); smooth distance on
    the distance, / max(|d|, h) with h = 2/1000 the spacing of the 1000^2 slice plane."""
    est = np.asarray(est, np.float64)
    ref = np.asarray(ref, np.float64)
    if kind == "winding":
        return np.abs(est - ref) / np.maximum(np.abs(ref), 1.0)
    if kind == "smoothdist":
        return np.abs(est - ref) / np.maximum(np.abs(ref), 2.0 / 1000.0)
    return np.abs(est - ref) / np.abs(ref)


def interp_loglog(x_target, xs, ys):
    """Linear interpolation of log(y) against log(x) at x_target (as in the paper's Fig. 4);
    returns (y, extrapolated)."""
    xs = np.asarray(xs, np.float64)
    ys = np.asarray(ys, np.float64)
    order = np.argsort(xs)
    lx, ly = np.log(xs[order]), np.log(ys[order])
    t = np.log(x_target)
    if t < lx[0] or t > lx[-1]:
        i = 0 if t < lx[0] else len(lx) - 2
        slope = (ly[i + 1] - ly[i]) / (lx[i + 1] - lx[i]) if lx[i + 1] != lx[i] else 0.0
        return float(np.exp(ly[i] + slope * (t - lx[i]))), True
    return float(np.exp(np.interp(t, lx, ly))), False


def tail_errors(rel):
    """Mean and 99th percentile of per-query relative errors (finite ones)."""
    r = np.asarray(rel, np.float64)
    r = r[np.isfinite(r)]
    return {"mean": float(r.mean()), "p99": float(np.percentile(r, 99))}


def error_stats(kind, est, ref):
    """Absolute and relative errors (relative as in rel_error) of an estimate: mean, median, max."""
    est = np.asarray(est, np.float64)
    ref = np.asarray(ref, np.float64)
    ok = np.isfinite(est)
    a = np.abs(est - ref)[ok]
    r = rel_error(kind, est, ref)[ok]
    return {"abs": {"mean": float(a.mean()), "median": float(np.median(a)), "max": float(a.max())},
            "rel": {"mean": float(r.mean()), "median": float(np.median(r)), "max": float(r.max())},
            "non_finite": int((~ok).sum()), "queries": int(est.size)}


def source_hash(paths):
    """Hash of the code of the kernel sources: comments and whitespace are dropped, so that only a
    change to the code itself marks a profile as stale."""
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


# the kernel and the tree layout it reads (the build writes the interleaved records and the guide)
EVAL_SOURCES = ["paper_2506_02219_gb300/csrc/sbh_eval_batched.cu", "paper_2506_02219_gb300/csrc/sbh_internal.cuh",
                "paper_2506_02219_gb300/csrc/sbh_learned.cuh", "paper_2506_02219_gb300/csrc/sbh_build.cu",
                "paper_2506_02219_gb300/csrc/sbh_build.cuh"]


def profiled_bytes(workload: str, key: str = "dram_bytes_per_query"):
    """Bytes per query of the estimator kernel (DRAM, or L2 with key l2_bytes_per_query) from the
    committed ncu summary, if the kernel sources still hash to what was profiled; else None."""
    path = os.path.join(ROOT, "profiles", f"k_stoch_batched_{workload}.md")
    if not os.path.exists(path):
        return None
    want = source_hash(EVAL_SOURCES)
    vals = {}
    for ln in open(path):
        if ln.startswith("<!-- ") and "=" in ln:
            k, v = ln[5:].strip().rstrip("->").strip().split("=", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != want or key not in vals:
        return None
    return float(vals[key])


def measured_hbm_gbs():
    """The measured HBM copy bandwidth (GB/s) of this machine's GPUs, or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def timed_ms(fn, dev, reps=3):
    """Median event-timed duration (ms) of fn on the current stream, after one untimed call, with
    L2 flushed (outside the events) before every timed call."""
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush_l2(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------------
def oracle_throughput(wl, seconds: float, S: int = 1):
    """Time the oracle on the host cores: its tree build over all sources plus its replay of a
    sample of queries sized to about `seconds` of work; returns (queries/s extrapolated to the full
    query set, cores used, description of the sample)."""
    import oracle
    kinds = {"coulomb": oracle.COULOMB, "winding": oracle.WINDING, "smoothdist": oracle.SMOOTHDIST}
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    tree = oracle.Tree(wl.points, wl.weights, wl.normals, leaf_size=wl.leaf_size, d=4)
    t_build = time.perf_counter() - t0
    nq = wl.queries.shape[0]
    rng = np.random.default_rng(5)
    pilot = min(nq, 8192)
    idx = rng.choice(nq, pilot, replace=False)
    t0 = time.perf_counter()
    tree.replay(wl.queries[idx], S=S, seed=7, kind=kinds[wl.kernel], softening=wl.softening, alpha=wl.alpha,
                query_index=idx)
    per_q = (time.perf_counter() - t0) / pilot
    n_sample = int(min(nq, max(pilot, (seconds - t_build) / max(per_q, 1e-9))))
    idx = rng.choice(nq, n_sample, replace=False)
    t0 = time.perf_counter()
    tree.replay(wl.queries[idx], S=S, seed=7, kind=kinds[wl.kernel], softening=wl.softening, alpha=wl.alpha,
                query_index=idx)
    t_replay = time.perf_counter() - t0
    t_full = t_build + t_replay * nq / n_sample
    desc = (f"oracle tree build over all {wl.points.shape[0]} sources ({t_build:.2f} s) + replay of "
            f"{n_sample} random queries of {nq} ({t_replay:.2f} s), replay time scaled linearly to all queries")
    return nq / t_full, cores, desc, t_full


# ------------------------------------------------------------------------------------------------
# the GPU arm
# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", local if world > 1 else 0)
    import paper_2506_02219_gb300 as sbh
    from paper_2506_02219_gb300 import _build
    _build.build()
    sbh.load_library()

    wl = workload_by_name(args.workload, rank)
    S, seed = args.S, 0x5BA7 + rank
    n, nq = wl.points.shape[0], wl.queries.shape[0]
    P = torch.from_numpy(wl.points).to(dev)
    M = torch.from_numpy(wl.weights).to(dev)
    N = torch.from_numpy(wl.normals).to(dev) if (wl.normals is not None and wl.kernel == "winding") else None
    Q = torch.from_numpy(wl.queries).to(dev)
    out = torch.empty(nq, dtype=torch.float32, device=dev)
    kk = _kernel_kwargs(wl)
    stream = torch.cuda.current_stream(dev)

    def step(keep):
        flush_l2(dev)
        s0 = torch.cuda.Event(enable_timing=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        tree = sbh.sbh_build(P, M, N, leaf_size=wl.leaf_size)
        e0.record(stream)
        sbh.sbh_eval(tree, Q, samples_per_subdomain=S, seed=seed, out=out, **kk)
        e1.record(stream)
        keep.append(tree)
        return s0, e0, e1

    keep = []
    for _ in range(args.warmup):
        step(keep)
    torch.cuda.synchronize()
    for t in keep:
        t.free()
    keep = []
    input_bytes = Q.numel() * 4 + P.numel() * 4 + M.numel() * 4 + (N.numel() * 4 if N is not None else 0)

    clocks = ClockSampler(local if world > 1 else 0)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = sbh.sbh_kernel_launches()
    evs = [step(keep) for _ in range(args.steps)]
    torch.cuda.synchronize()
    barrier(world)
    launches = sbh.sbh_kernel_launches() - launches0
    clk = clocks.stop()
    # each step from the start of its build to the end of its evaluation (the L2 flush before it untimed)
    step_ms = float(np.mean([s0.elapsed_time(e1) for s0, _, e1 in evs]))
    eval_ms = float(np.mean([e0.elapsed_time(e1) for _, e0, e1 in evs]))
    for t in keep:
        t.free()
    max_s = reduce_max(step_ms * args.steps / 1e3, world, dev)
    value = weak_scaling_value(nq * args.steps, world, max_s)

    # end to end through the public API with pinned host buffers
    Ph = torch.from_numpy(wl.points).pin_memory()
    Mh = torch.from_numpy(wl.weights).pin_memory()
    Nh = torch.from_numpy(wl.normals).pin_memory() if N is not None else None
    Qh = torch.from_numpy(wl.queries).pin_memory()
    Oh = torch.empty(nq, dtype=torch.float32).pin_memory()

    def e2e_step():
        # one C-ABI call on host buffers: uploads, build, chunked evaluation and download pipelined
        sbh.sbh_solve_host(Ph, Mh, Qh, normals=Nh, leaf_size=wl.leaf_size, samples_per_subdomain=S, seed=seed,
                           out=Oh, **kk)

    for _ in range(2):
        e2e_step()
    barrier(world)
    ts = time.perf_counter()
    k_e2e = max(3, args.steps // 2)
    for _ in range(k_e2e):
        e2e_step()
    e2e_s = reduce_max((time.perf_counter() - ts), world, dev)
    h2d = Ph.numel() * 4 + Mh.numel() * 4 + (Nh.numel() * 4 if Nh is not None else 0) + Qh.numel() * 4
    e2e = {"value": weak_scaling_value(nq * k_e2e, world, e2e_s), "unit": "queries/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(nq * 4), "api": "sbh_solve_host"}

    result = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": max_s * 1e3 / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
              "config": {"workload": wl.name, "sources": int(n), "queries": int(nq), "kernel": wl.kernel,
                         "samples_per_subdomain": S, "leaf_size": wl.leaf_size, "step": "sbh_build + sbh_eval",
                         "l2": f"{L2_NOTE}; inputs {input_bytes / 2**20:.0f} MiB per step, L2 129 MiB",
                         "parallelism": f"replicas x{world}"},
              "e2e": e2e, "gpu_launches": int(launches), "gpu_launches_per_step": launches / args.steps,
              "clocks": clk, "eval_ms_per_step": eval_ms, "build_ms_per_step": step_ms - eval_ms}

    if rank == 0:
        # work of one estimator launch, counted by the same traversal
        tree = sbh.sbh_build(P, M, N, leaf_size=wl.leaf_size)
        cnt = sbh.sbh_eval_count(tree, Q, samples_per_subdomain=S, seed=seed, **kk)
        c = np.array([cnt["terms"], cnt["records"], cnt["decisions"], cnt["cdf_reads"]], np.float64)
        flops = c[0] * FLOPS_PER_TERM[wl.kernel]
        sms = int(torch.cuda.get_device_properties(dev).multi_processor_count)
        sm_mhz, clk_src = peak_clock_mhz(clk)
        peak = fp32_peak_tflops(sms, sm_mhz)
        achieved = flops / (eval_ms / 1e3) / 1e12
        traffic_pq = profiled_bytes(args.workload)
        l2_pq = profiled_bytes(args.workload, "l2_bytes_per_query")
        hbm_peak = measured_hbm_gbs()
        memory = {}
        if traffic_pq is not None:
            gbs = traffic_pq * nq / (eval_ms / 1e3) / 1e9
            memory["dram"] = {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "peak_basis": "measured (MEASURED_PEAKS.json)",
                              "frac": gbs / hbm_peak if hbm_peak else None, "bytes_per_query": traffic_pq}
        if l2_pq is not None:
            memory["l2"] = {"achieved_gbs": l2_pq * nq / (eval_ms / 1e3) / 1e9, "bytes_per_query": l2_pq,
                            "note": "L2 sectors of one ncu capture (all sources) per query; no measured L2 peak"}
        result["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                              "frac": achieved / peak,
                              "traffic": (traffic_pq * nq) if traffic_pq is not None else None,
                              "traffic_source": (f"ncu capture summarised in profiles/k_stoch_batched_{args.workload}.md "
                                                 f"(dram__bytes_read.sum + dram__bytes_write.sum per query x queries), "
                                                 f"used because its kernel-source hash {source_hash(EVAL_SOURCES)} "
                                                 f"matches this build") if traffic_pq is not None else
                                                "none: no ncu capture of this kernel source",
                              "memory": memory,
                              "kernel": "k_stoch_batched", "terms_per_query": c[0] / nq,
                              "records_per_query": c[1] / nq, "decisions_per_query": c[2] / nq,
                              "flops_per_term": FLOPS_PER_TERM[wl.kernel],
                              "sm_count": sms, "sm_mhz": sm_mhz,
                              "peak_basis": (f"{sms} SMs (queried from the device) x {FP32_LANES_PER_SM} FP32 lanes x "
                                             f"2 flop x {sm_mhz:.0f} MHz ({clk_src})")}
        # the adjoint (value and query gradient under the same random stream)
        g_out = torch.empty(nq, dtype=torch.float32, device=dev)
        g_grad = torch.empty((nq, 3), dtype=torch.float32, device=dev)
        sbh.sbh_eval_grad(tree, Q, samples_per_subdomain=S, seed=seed, out=g_out, grad=g_grad, **kk)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush_l2(dev)
        a0.record(stream)
        sbh.sbh_eval_grad(tree, Q, samples_per_subdomain=S, seed=seed, out=g_out, grad=g_grad, **kk)
        a1.record(stream)
        a1.synchronize()
        result["adjoint"] = {"ms": a0.elapsed_time(a1), "queries_per_s": nq / (a0.elapsed_time(a1) / 1e3)}
        if args.learned_near is not None:
            # the learned child proposal alone at one gate: trained, then timed at S = 1 (no error sweep)
            net = sbh.sbh_mlp_create(1)
            lo, hi = wl.points.min(0), wl.points.max(0)
            qt = np.random.default_rng(5).uniform(lo - 0.05 * (hi - lo), hi + 0.05 * (hi - lo),
                                                  (1024, 3)).astype(np.float32)
            sbh.sbh_mlp_train(net, tree, torch.from_numpy(qt).to(dev), near=args.learned_near, steps=300, lr=3e-3,
                              **kk)
            lout = sbh.sbh_eval_learned(tree, net, Q, seed=seed, near=args.learned_near, **kk)
            lms = timed_ms(lambda: sbh.sbh_eval_learned(tree, net, Q, seed=seed, near=args.learned_near, out=lout,
                                                        **kk), dev, 3)
            result["learned"] = {"near": args.learned_near, "ms": lms, "queries_per_s": nq / (lms / 1e3)}
        if not args.no_equal_error:
            result["equal_error"] = equal_error(sbh, wl, tree, P, M, N, Q, S, seed, eval_ms, dev)
            summary = {"ordered": {"queries": wl.name,
                                   "speedup_vs_bh_at_equal_median_error":
                                       result["equal_error"]["speedup_vs_bh_at_equal_median_error"]}}
            if args.workload == "winding":
                # the same sources with as many queries drawn uniformly in their bounding box, unsorted
                from paper_2506_02219_gb300 import workloads as W
                wr = W.winding_ellipsoids_random(seed=W.BASE_SEED + 1 + 1000 * rank)
                Qr = torch.from_numpy(wr.queries).to(dev)
                rnd = equal_error_compact(sbh, wl, tree, P, M, N, Qr, S, seed, dev)
                rnd["queries"] = wr.name
                result["equal_error_random_order"] = rnd
                summary["random_order"] = {"queries": wr.name,
                                           "speedup_vs_bh_at_equal_median_error":
                                               rnd["speedup_vs_bh_at_equal_median_error"]}
                del Qr
                # the slice-plane configuration (Coulomb and smooth distance), compact
                sp = slice_plane_compact(sbh, seed, dev, rank)
                result["slice_plane"] = sp
                # the batched configuration, compact (its own line: --workload batched)
                b = batched_measure(sbh, dev, 5, 3)
                result["batched"] = {"ms_per_step": b["ms_per_step"], "queries_per_s": b["queries_per_s"],
                                     "config": b["config"], "autotune_best": b["autotune"]["best"],
                                     "build_s_all_sets": b["build_s_all_sets"], "adjoint": b["adjoint"]}
                for kind in ("coulomb", "smoothdist"):
                    summary[f"slice_plane_{kind}"] = {"queries": f"{kind}_shapes_4194304src_1000x1000plane",
                                                      "speedup_vs_bh_at_equal_median_error":
                                                          sp[kind]["speedup_vs_bh_at_equal_median_error"]}
            result["equal_error_summary"] = summary
        tree.free()
        if world == 1 and not args.no_cpu_baseline:
            v, cores, desc, _ = oracle_throughput(wl, args.cpu_seconds, S)
            result["cpu_baseline"] = {"value": v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                                      "sample": desc}
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def equal_error_compact(sbh, wl, tree, P, M, N, Q, S, seed, dev,
                        thetas=(3.0, 2.0, 1.5, 1.2, 1.0, 0.8, 0.67, 0.5, 0.4)):
    """The estimator at S against the project's Barnes-Hut on one query set: estimator time and
    median / mean / p99 relative error (65536 sampled queries against the FP64-accumulated GPU brute
    force), the Barnes-Hut theta sweep with and without warp voting, and the Barnes-Hut time at the
    estimator's median error (log-log interpolation, the faster voting mode)."""
    import torch
    nq = Q.shape[0]
    kk = _kernel_kwargs(wl)
    g = torch.Generator(device="cpu").manual_seed(13)
    idx = torch.randperm(nq, generator=g)[: min(nq, 65536)].sort().values.to(dev)
    Qs = Q[idx].contiguous()
    ref = sbh.sbh_eval_brute(P, M, Qs, normals=N, fp64_accum=True, **kk).cpu().numpy()
    out = sbh.sbh_eval(tree, Q, samples_per_subdomain=S, seed=seed, **kk)
    ms = timed_ms(lambda: sbh.sbh_eval(tree, Q, samples_per_subdomain=S, seed=seed, out=out, **kk), dev, 3)
    rel = rel_error(wl.kernel, out[idx].cpu().numpy(), ref)
    err = float(np.median(rel))
    bh_out = torch.empty(nq, dtype=torch.float32, device=dev)
    sweep = []
    for vote in (True, False):
        for theta in thetas:
            t = timed_ms(lambda: sbh.sbh_eval_bh(tree, Q, theta=theta, warp_vote=vote, out=bh_out, **kk), dev, 2)
            e = rel_error(wl.kernel, sbh.sbh_eval_bh(tree, Qs, theta=theta, warp_vote=vote, **kk).cpu().numpy(), ref)
            sweep.append({"theta": theta, "warp_vote": vote, "ms": t, "median_rel_err": float(np.median(e))})
    best = None
    for vote in (True, False):
        pts = [(s["median_rel_err"], s["ms"]) for s in sweep if s["warp_vote"] == vote and s["median_rel_err"] > 0]
        t_bh, extrap = interp_loglog(err, [p[0] for p in pts], [p[1] for p in pts])
        if best is None or t_bh < best[0]:
            best = (t_bh, extrap, vote)
    return {"S": S, "ms": ms, "median_rel_err": err, "tail": tail_errors(rel), "bh_sweep": sweep,
            "bh_ms_at_equal_error": best[0], "bh_warp_vote": best[2], "extrapolated": best[1],
            "speedup_vs_bh_at_equal_median_error": best[0] / ms,
            "error_reference": "GPU brute force with FP64 tile accumulation on 65536 random queries"}


def slice_plane_compact(sbh, seed, dev, rank=0, s_max=4, config_thetas=(0.3, 0.5, 0.8)):
    """The slice-plane configuration: 2^22 samples on a union of 8 ellipsoids and 4 boxes, 1000^2
    queries on the plane z = 0, for the Coulomb kernel (area weights) and the smooth distance
    (alpha = 200, unit weights; the same samples and queries). Per kernel: the tree build, the
    estimator at S = 1 ... s_max (event-timed, median relative error on 65536 sampled queries), the
    project's Barnes-Hut at the configuration's thetas, and the compact equal-error comparison at
    S = 1 (equal_error_compact)."""
    import dataclasses
    import torch
    from paper_2506_02219_gb300 import workloads as W
    base = W.slice_plane_shapes(kernel="coulomb", seed=W.BASE_SEED + 2 + 1000 * rank)
    P = torch.from_numpy(base.points).to(dev)
    Q = torch.from_numpy(base.queries).to(dev)
    nq = Q.shape[0]
    g = torch.Generator(device="cpu").manual_seed(13)
    idx = torch.randperm(nq, generator=g)[: min(nq, 65536)].sort().values.to(dev)
    Qs = Q[idx].contiguous()
    res = {"sources": base.points.shape[0], "queries": nq}
    for kind in ("coulomb", "smoothdist"):
        w = base.weights if kind == "coulomb" else np.ones_like(base.weights)
        wl = dataclasses.replace(base, weights=w, kernel=kind, name=f"{kind}_shapes_{base.points.shape[0]}src_1000x1000plane")
        kk = _kernel_kwargs(wl)
        M = torch.from_numpy(wl.weights).to(dev)
        build_ms = timed_ms(lambda: sbh.sbh_build(P, M, None, leaf_size=wl.leaf_size).free(), dev, 2)
        tree = sbh.sbh_build(P, M, None, leaf_size=wl.leaf_size)
        ref = sbh.sbh_eval_brute(P, M, Qs, fp64_accum=True, **kk).cpu().numpy()
        rows = []
        for S in range(1, s_max + 1):
            out = sbh.sbh_eval(tree, Q, samples_per_subdomain=S, seed=seed, **kk)
            ms = timed_ms(lambda: sbh.sbh_eval(tree, Q, samples_per_subdomain=S, seed=seed, out=out, **kk), dev, 3)
            e = rel_error(kind, out[idx].cpu().numpy(), ref)
            rows.append({"S": S, "ms": ms, "median_rel_err": float(np.median(e))})
        bh = []
        bh_out = torch.empty(nq, dtype=torch.float32, device=dev)
        for theta in config_thetas:
            for vote in (True, False):
                t = timed_ms(lambda: sbh.sbh_eval_bh(tree, Q, theta=theta, warp_vote=vote, out=bh_out, **kk), dev, 2)
                e = rel_error(kind, sbh.sbh_eval_bh(tree, Qs, theta=theta, warp_vote=vote, **kk).cpu().numpy(), ref)
                bh.append({"theta": theta, "warp_vote": vote, "ms": t, "median_rel_err": float(np.median(e))})
        eq = equal_error_compact(sbh, wl, tree, P, M, None, Q, 1, seed, dev)
        res[kind] = {"build_ms": build_ms, "estimator": rows, "bh_config_thetas": bh,
                     "bh_ms_at_equal_error": eq["bh_ms_at_equal_error"], "bh_warp_vote": eq["bh_warp_vote"],
                     "extrapolated": eq["extrapolated"],
                     "speedup_vs_bh_at_equal_median_error": eq["speedup_vs_bh_at_equal_median_error"]}
        if kind == "coulomb":
            # the learned child proposal at gate 0.25 against the mass estimator at the same median error
            ln = learned_proposal(sbh, wl, tree, Q, idx, ref, seed, kk, lambda fn, reps: timed_ms(fn, dev, reps), 0.25)
            m_ms, m_ex = interp_loglog(ln["median_rel_err"], [r["median_rel_err"] for r in rows], [r["ms"] for r in rows])
            res[kind]["learned_proposal_near0.25"] = {"ms": ln["ms"], "median_rel_err": ln["median_rel_err"],
                                                      "mass_ms_at_equal_error": m_ms, "mass_extrapolated": m_ex,
                                                      "speedup_vs_mass": m_ms / ln["ms"]}
        tree.free()
    return res


def equal_error(sbh, wl, tree, P, M, N, Q, S, seed, eval_ms, dev):
    """Median relative error of the estimator (S = 1) against the exact sum, and the Barnes-Hut
    theta sweep (time per query set, median error); the Barnes-Hut time at the estimator's median
    error by log-log interpolation, as in the paper's Fig. 4."""
    import torch
    nq = Q.shape[0]
    kk = _kernel_kwargs(wl)
    g = torch.Generator(device="cpu").manual_seed(11)
    idx = torch.randperm(nq, generator=g)[: min(nq, 65536)].sort().values.to(dev)
    Qs = Q[idx].contiguous()
    ref = sbh.sbh_eval_brute(P, M, Qs, normals=N, fp64_accum=True, **kk).cpu().numpy()
    out = sbh.sbh_eval(tree, Q, samples_per_subdomain=S, seed=seed, **kk)
    err_s = float(np.median(rel_error(wl.kernel, out[idx].cpu().numpy(), ref)))
    stats_s = error_stats(wl.kernel, out[idx].cpu().numpy(), ref)
    tail_s = tail_errors(rel_error(wl.kernel, out[idx].cpu().numpy(), ref))

    def timed(fn, reps=3):
        return timed_ms(fn, dev, reps)

    extra = {}
    for s2 in (2, 3, 4, 8, 16, 32):
        o2 = sbh.sbh_eval(tree, Q, samples_per_subdomain=s2, seed=seed, **kk)
        r2 = rel_error(wl.kernel, o2[idx].cpu().numpy(), ref)
        extra[f"S{s2}"] = {"ms": timed(lambda: sbh.sbh_eval(tree, Q, samples_per_subdomain=s2, seed=seed, out=o2, **kk), 2),
                           "median_rel_err": float(np.median(r2)), "tail": tail_errors(r2)}
    # the paper's variants (supplemental: roulette off / fixed 1/2; Algorithm 2's uniform path
    # index; identical seeding across queries) and the one-thread-per-query schedule, at S = 1
    variants = {}
    for name, opt in (("roulette_off", sbh.eval_opts(rr=1)), ("roulette_half", sbh.eval_opts(rr=2)),
                      ("uniform_path_index", sbh.eval_opts(sampling=1)), ("coherent_seed", sbh.eval_opts(seed_mode=1)),
                      ("thread_per_query", sbh.eval_opts(schedule=1))):
        ov = sbh.sbh_eval(tree, Q, samples_per_subdomain=S, seed=seed, opts=opt, **kk)
        ms = timed(lambda: sbh.sbh_eval(tree, Q, samples_per_subdomain=S, seed=seed, opts=opt, out=ov, **kk), 2)
        err = float(np.median(rel_error(wl.kernel, ov[idx].cpu().numpy(), ref)))
        variants[name] = {"ms": ms, "median_rel_err": err}
    bh_out = torch.empty(nq, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    sbh.sbh_eval_bh(tree, Q[:1], theta=0.5, **kk)  # builds the 8-ary tree
    torch.cuda.synchronize()
    bh_build_ms = (time.perf_counter() - t0) * 1e3
    sweep = []
    for vote in (True, False):
        for theta in (3.0, 2.0, 1.5, 1.2, 1.0, 0.8, 0.67, 0.5, 0.4, 0.3, 0.25):
            ms = timed(lambda: sbh.sbh_eval_bh(tree, Q, theta=theta, warp_vote=vote, out=bh_out, **kk))
            e = sbh.sbh_eval_bh(tree, Qs, theta=theta, warp_vote=vote, **kk).cpu().numpy()
            re_bh = rel_error(wl.kernel, e, ref)
            sweep.append({"theta": theta, "warp_vote": vote, "ms": ms,
                          "median_rel_err": float(np.median(re_bh)), "tail": tail_errors(re_bh)})
    def bh_time_at(err, stat="median"):
        best = None
        for vote in (True, False):
            pts = [((s["median_rel_err"] if stat == "median" else s["tail"][stat]), s["ms"])
                   for s in sweep if s["warp_vote"] == vote]
            pts = [p for p in pts if p[0] > 0]
            t_bh, extrap = interp_loglog(err, [p[0] for p in pts], [p[1] for p in pts])
            if best is None or t_bh < best[0]:
                best = (t_bh, extrap, vote)
        return best

    best = bh_time_at(err_s)
    # the mass-proportional estimator's time at a given error, from its S = 1 .. 4 rows
    mass_pts = [(err_s, eval_ms)] + [(v["median_rel_err"], v["ms"]) for v in extra.values()]
    for near in LEARNED_NEARS:
        learned = learned_proposal(sbh, wl, tree, Q, idx, ref, seed, kk, timed, near)
        t_mass, extrap_m = interp_loglog(learned["median_rel_err"], [p[0] for p in mass_pts], [p[1] for p in mass_pts])
        learned["mass_ms_at_equal_error"] = t_mass
        learned["mass_extrapolated"] = extrap_m
        learned["speedup_vs_mass"] = t_mass / learned["ms"]
        for stat in ("mean", "p99"):  # the same comparison on the mean and the 99th percentile of the errors
            pts = [(tail_s[stat], eval_ms)] + \
                  [(v["tail"][stat], v["ms"]) for v in extra.values()]
            t_m, ex_m = interp_loglog(learned["tail"][stat], [p[0] for p in pts], [p[1] for p in pts])
            learned[f"speedup_vs_mass_at_equal_{stat}_error"] = t_m / learned["ms"]
            learned[f"mass_extrapolated_{stat}"] = ex_m
            learned[f"speedup_vs_bh_at_equal_{stat}_error"] = bh_time_at(learned["tail"][stat], stat)[0] / learned["ms"]
        variants[f"learned_proposal_near{near:g}"] = learned
    for v in list(extra.values()) + list(variants.values()):
        t_bh, extrap, _ = bh_time_at(v["median_rel_err"])
        v["bh_ms_at_equal_error"] = t_bh
        v["speedup_vs_bh"] = t_bh / v["ms"]
    return {"stochastic": {"S": S, "ms": eval_ms, "median_rel_err": err_s, "errors": stats_s, **extra},
            "variants": variants,
            "bh_sweep": sweep, "bh_tree_build_ms": bh_build_ms,
            "bh_ms_at_equal_error": best[0], "bh_warp_vote": best[2], "extrapolated": best[1],
            "speedup_vs_bh_at_equal_median_error": best[0] / eval_ms,
            "speedup_vs_bh_at_equal_mean_error": bh_time_at(tail_s["mean"], "mean")[0] / eval_ms,
            "speedup_vs_bh_at_equal_p99_error": bh_time_at(tail_s["p99"], "p99")[0] / eval_ms,
            "error_reference": "GPU brute force with FP64 tile accumulation on 65536 random queries",
            "time_basis": "evaluation kernels only, trees prebuilt (the paper excludes building)"}


LEARNED_NEARS = (0.25, 0.5, 1.0)  # gates of the learned proposal, in cell diagonals


def learned_proposal(sbh, wl, tree, Q, idx, ref, seed, kk, timed, near):
    """Train the learned child proposal on 1024 random queries in the sources' bounding box (the
    residuals the estimator's own paths meet there), then time it at S = 1 on the full query set."""
    import torch
    lo, hi = wl.points.min(0), wl.points.max(0)
    qt = np.random.default_rng(5).uniform(lo - 0.05 * (hi - lo), hi + 0.05 * (hi - lo), (1024, 3)).astype(np.float32)
    net = sbh.sbh_mlp_create(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = sbh.sbh_mlp_train(net, tree, torch.from_numpy(qt).to(Q.device), near=near, steps=300, lr=3e-3, **kk)
    train_s = time.perf_counter() - t0
    out = sbh.sbh_eval_learned(tree, net, Q, seed=seed, near=near, **kk)
    ms = timed(lambda: sbh.sbh_eval_learned(tree, net, Q, seed=seed, near=near, out=out, **kk), 2)
    rl = rel_error(wl.kernel, out[idx].cpu().numpy(), ref)
    err = float(np.median(rl))
    return {"ms": ms, "median_rel_err": err, "tail": tail_errors(rl), "near": near, "train_s": train_s,
            "train": {"queries": 1024, "adam_steps": 300, "lr": 3e-3, "loss_first": float(losses[0]),
                      "loss_last": float(losses[-1])},
            "scorer": "tensor cores (mma.sync m16n8k16, FP16 operands, FP32 accumulation)"}


# ------------------------------------------------------------------------------------------------
# the reference arm: the CPU oracle as it stands
# ------------------------------------------------------------------------------------------------
def oracle_full_step(wl, S: int = 1):
    """One whole step of the oracle on the host cores: its tree build over all sources and its
    replay of every query. Returns (seconds, cores)."""
    import oracle
    kinds = {"coulomb": oracle.COULOMB, "winding": oracle.WINDING, "smoothdist": oracle.SMOOTHDIST}
    t0 = time.perf_counter()
    tree = oracle.Tree(wl.points, wl.weights, wl.normals, leaf_size=wl.leaf_size, d=4)
    tree.replay(wl.queries, S=S, seed=7, kind=kinds[wl.kernel], softening=wl.softening, alpha=wl.alpha)
    return time.perf_counter() - t0, oracle.max_threads()


REFERENCE_BUDGET_S = 200.0  # the timed steps of the reference arm stop short of this


def run_reference(args):
    """The CPU oracle as it stands, timed on the host cores on the same workload: every timed step
    is a whole step (tree build over all sources + replay of every query), measured. The first
    warm-up is a whole step too and sizes the run: if K whole steps would take longer than
    REFERENCE_BUDGET_S, fewer are timed (and reported as the steps taken); the other warm-ups replay
    a bounded sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = workload_by_name(args.workload, 0)
    t_first, cores = oracle_full_step(wl, args.S)
    for _ in range(args.warmup - 1):
        oracle_throughput(wl, 2.0, args.S)
    steps = int(min(args.steps, max(1, REFERENCE_BUDGET_S // t_first)))
    ts = [oracle_full_step(wl, args.S)[0] for _ in range(steps)]
    nq = int(wl.queries.shape[0])
    value = nq * steps / float(np.sum(ts))
    desc = (f"whole steps: oracle tree build over all {wl.points.shape[0]} sources + replay of all {nq} queries, "
            f"{steps} timed (first warm-up step {t_first:.2f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
            "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(ts)) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "sources": int(wl.points.shape[0]), "queries": nq,
                       "kernel": wl.kernel, "samples_per_subdomain": args.S, "leaf_size": wl.leaf_size,
                       "step": "oracle tree build + Algorithm 2 replay of every query (FP64, CPU)"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if steps != args.steps:
        line["steps_requested"] = args.steps
    print(json.dumps(line), flush=True)


def batched_sets(rank: int = 0, n_sets: int = 64):
    """64 independent problems: sources log-uniform in [2^10, 2^20] (shape unions with area weights),
    queries log-uniform in [2^8, 2^18] uniform in each set's bounding box."""
    from paper_2506_02219_gb300 import workloads as W
    rng = np.random.default_rng(W.BASE_SEED + 3 + 1000 * rank)
    sets = []
    for i in range(n_sets):
        n = int(2 ** rng.uniform(10, 20))
        nq = int(2 ** rng.uniform(8, 18))
        p, w, _ = W.shape_union(n, int(rng.integers(1 << 30)), n_ellipsoids=4, n_boxes=2)
        lo, hi = p.min(0), p.max(0)
        q = (lo + rng.random((nq, 3)) * (hi - lo)).astype(np.float32)
        sets.append((p, w, q))
    return sets


BATCHED_KERNEL = "smoothdist"  # smooth distance (alpha = 200, unit weights) over the batched sets


def batched_adjoint(sbh, p, w, q, tree, S, seed, dev):
    """The adjoint on one set: time of sbh_eval_grad (value and d/dq under the estimator's stream),
    its median relative error against the GPU brute-force gradient (FP64 accumulation), and its
    median relative gap to central differences (h = 1e-4) of the estimate with the roulette off,
    where the frozen-path derivative is the derivative of the estimate."""
    import torch
    P, M, Q = (torch.from_numpy(x).to(dev) for x in (p, w, q))
    kk = dict(kernel=BATCHED_KERNEL, alpha=200.0)
    out, grad = sbh.sbh_eval_grad(tree, Q, samples_per_subdomain=S, seed=seed, **kk)
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        flush_l2(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sbh.sbh_eval_grad(tree, Q, samples_per_subdomain=S, seed=seed, out=out, grad=grad, **kk)
        e1.record()
        ts.append((e0, e1))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ts]))
    _, gref = sbh.sbh_eval_brute_grad(P, M, Q, **kk)
    g, gr = grad.double().cpu().numpy(), gref.double().cpu().numpy()
    ok = np.all(np.isfinite(g), axis=1) & np.all(np.isfinite(gr), axis=1)
    err = np.linalg.norm(g - gr, axis=1)[ok] / np.maximum(np.linalg.norm(gr, axis=1)[ok], 1e-30)
    # central differences of the estimate along each axis, roulette off
    o = sbh.eval_opts(rr=1)
    _, g1 = sbh.sbh_eval_grad(tree, Q, samples_per_subdomain=S, seed=seed, opts=o, **kk)
    h = 1e-4
    fd = torch.empty_like(g1)
    for a in range(3):
        dq = torch.zeros(3, device=dev)
        dq[a] = h
        fp = sbh.sbh_eval(tree, (Q + dq).contiguous(), samples_per_subdomain=S, seed=seed, opts=o, **kk)
        fm = sbh.sbh_eval(tree, (Q - dq).contiguous(), samples_per_subdomain=S, seed=seed, opts=o, **kk)
        fd[:, a] = (fp.double() - fm.double()).float() / (2 * h)
    g1n, fdn = g1.double().cpu().numpy(), fd.double().cpu().numpy()
    ok1 = np.all(np.isfinite(g1n), axis=1) & np.all(np.isfinite(fdn), axis=1)
    gap = np.linalg.norm(g1n - fdn, axis=1)[ok1] / np.maximum(np.linalg.norm(g1n, axis=1)[ok1], 1e-30)
    return {"set_sources": int(p.shape[0]), "set_queries": int(q.shape[0]), "S": S, "ms": ms,
            "queries_per_s": q.shape[0] / (ms / 1e3),
            "median_rel_err_vs_brute_grad": float(np.median(err)), "finite_fraction": float(ok.mean()),
            "median_rel_gap_vs_central_fd_roulette_off": float(np.median(gap)), "fd_h": h}


def batched_measure(sbh, dev, steps: int, warmup: int):
    """Many independent source/query sets (smooth distance) in one persistent, graph-captured launch;
    S and leaf size from the autotuner (on the largest set, the most efficient: smallest time x
    error^2). A step is one replay of the captured launch (the trees are built once, their build
    time is reported). Then the adjoint on the largest set against the brute-force gradient and
    finite differences. Returns the measurements as a dict."""
    import torch
    from paper_2506_02219_gb300 import autotune
    sets = [(p, np.ones_like(w), q) for p, w, q in batched_sets()]
    big = max(range(len(sets)), key=lambda i: sets[i][0].shape[0])
    p, w, q = sets[big]
    tune = autotune.autotune(torch.from_numpy(p).to(dev), torch.from_numpy(w).to(dev), torch.from_numpy(q).to(dev),
                             BATCHED_KERNEL, leaf_sizes=(1, 2, 4), samples=(1, 2), schedules=(0,))
    leaf, S = tune["best"]["leaf_size"], tune["best"]["S"]
    t0 = time.perf_counter()
    trees, Qs = [], []
    for p, w, q in sets:
        trees.append(sbh.sbh_build(torch.from_numpy(p).to(dev), torch.from_numpy(w).to(dev), leaf_size=leaf))
        Qs.append(torch.from_numpy(q).to(dev))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    plan = sbh.sbh_multi_plan_create(trees, Qs, BATCHED_KERNEL, S, seed=0x5BA7)
    graph = sbh.capture_multi(plan)
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = sbh.sbh_kernel_launches()
    evs = []
    for _ in range(steps):
        flush_l2(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    # graph replays launch the captured kernels without passing through the library's counter
    launches = sbh.sbh_kernel_launches() - launches0 + steps * graph.sbh_kernels
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    total_q = sum(int(q.shape[0]) for q in Qs)
    adj = batched_adjoint(sbh, *sets[big], trees[big], S, 0x5BA7, dev)
    return {"ms_per_step": ms, "queries_per_s": total_q / (ms / 1e3),
            "config": {"workload": f"batched_64sets_{BATCHED_KERNEL}", "sets": len(sets),
                       "sources": int(sum(s[0].shape[0] for s in sets)), "queries": total_q,
                       "kernel": BATCHED_KERNEL, "alpha": 200.0,
                       "samples_per_subdomain": S, "leaf_size": leaf,
                       "step": "one replay of the graph-captured multi-set launch", "l2": L2_NOTE},
            "build_s_all_sets": build_s, "autotune": tune, "adjoint": adj, "clocks": clk, "gpu_launches": launches}


def run_batched(args):
    """The batched configuration's own bench line (batched_measure)."""
    import torch
    import paper_2506_02219_gb300 as sbh
    from paper_2506_02219_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    r = batched_measure(sbh, dev, args.steps, args.warmup)
    print(json.dumps({"metric": METRIC, "value": r["queries_per_s"], "unit": "queries/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                      "data": "synthetic", "config": r["config"], "build_s_all_sets": r["build_s_all_sets"],
                      "autotune": r["autotune"], "adjoint": r["adjoint"], "clocks": r["clocks"],
                      "gpu_launches": r["gpu_launches"]}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="winding",
                    choices=["winding", "winding_random", "cube", "slice_coulomb", "slice_smoothdist", "far_coulomb",
                             "batched"])
    ap.add_argument("--S", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-equal-error", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--learned-near", type=float, default=None,
                    help="also train the learned proposal and time it alone at this gate (cell diagonals)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
