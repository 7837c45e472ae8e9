"""Autotuner for the estimator's launch parameters.

It measures, on the caller's own data, every combination of
  leaf size (tree build), samples per subdomain S, and schedule (0: warp task batches, 1: one
  thread per query),
the GPU time of sbh_eval over the query set and its median relative error against the exact sum on
a sample of queries (GPU brute force with FP64 accumulation), and picks the fastest combination
whose median error meets a target -- or, without a target, the most efficient one (smallest
time x error^2: the work to reach a fixed error, since the estimator's error falls as 1/sqrt(S)).
Everything runs in the library's kernels; this module only times calls and compares numbers.
"""
from __future__ import annotations

import itertools

import numpy as np


def _median_rel_err(kind, est, ref):
    est = np.asarray(est, np.float64)
    ref = np.asarray(ref, np.float64)
    if kind == "winding":
        return float(np.median(np.abs(est - ref) / np.maximum(np.abs(ref), 1.0)))
    if kind == "smoothdist":
        return float(np.median(np.abs(est - ref) / np.maximum(np.abs(ref), 1e-3)))
    return float(np.median(np.abs(est - ref) / np.abs(ref)))


def autotune(points, weights, queries, kernel: str = "coulomb", normals=None, target_median_rel_err=None,
             leaf_sizes=(1, 2, 4), samples=(1, 2, 4), schedules=(0, 1), n_err_queries: int = 8192,
             softening: float = 1e-3, alpha: float = 200.0, seed: int = 0, reps: int = 3) -> dict:
    """Measure every configuration and return {"best": {...}, "table": [...]}. Tensors are CUDA,
    float32, as for sbh_build / sbh_eval."""
    import torch

    import paper_2506_02219_gb300 as sbh

    nq = queries.shape[0]
    g = torch.Generator(device="cpu").manual_seed(1234)
    idx = torch.randperm(nq, generator=g)[: min(nq, n_err_queries)].to(queries.device)
    ref = sbh.sbh_eval_brute(points, weights, queries[idx].contiguous(), kernel, normals=normals, fp64_accum=True,
                             softening=softening, alpha=alpha).cpu().numpy()
    out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    table = []
    for leaf in leaf_sizes:
        tree = sbh.sbh_build(points, weights, normals, leaf_size=leaf)
        for S, sched in itertools.product(samples, schedules):
            o = sbh.eval_opts(schedule=sched)

            def run():
                sbh.sbh_eval(tree, queries, kernel, S, seed, opts=o, out=out, softening=softening, alpha=alpha)

            run()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                run()
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            err = _median_rel_err(kernel, out[idx].cpu().numpy(), ref)
            table.append({"leaf_size": leaf, "S": S, "schedule": sched, "ms": float(np.median(ts)),
                          "median_rel_err": err})
        tree.free()
    return {"best": select(table, target_median_rel_err), "table": table}


def select(table, target_median_rel_err=None) -> dict:
    """The configuration to use from measured rows {"ms", "median_rel_err", ...}: with a target,
    the fastest row that meets it (the most accurate row if none does); without one, the row
    with the smallest ms x error^2 (the time to reach a fixed error, the error falling as
    1/sqrt(S)). Ties keep the first row in table order."""
    if not table:
        raise ValueError("no measured configuration")
    if target_median_rel_err is not None:
        ok = [r for r in table if r["median_rel_err"] <= target_median_rel_err]
        return min(ok, key=lambda r: r["ms"]) if ok else min(table, key=lambda r: r["median_rel_err"])
    return min(table, key=lambda r: r["ms"] * r["median_rel_err"] ** 2)
