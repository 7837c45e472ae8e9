"""Study: the estimator against Barnes-Hut on a Table-1-like case, under each reading of the paper.

Run as ``python tests/study_readings.py [--n 32768] [--seeds 8]``. It prints one row per
(reading, query set), all from the FP64 CPU oracle:

- the case: one closed surface (a random ellipsoid, area-uniform samples) rescaled into
  [-1, 1]^3, masses summing to 1, the Coulomb kernel (Sec. 4.2, Table 1);
- queries: 4096 points of the 100^3 grid over [-1, 1]^3 and 4096 uniform points in the cube;
- est_med: the median over queries and seeds of |F_1(q) - F(q)| at S = 1 (Algorithm 2);
- est_work: kernel terms per query (control variates plus every swap's children and node);
- bias: the median over 256 queries of |E[F_1(q)] - F(q)|, E by exact enumeration;
- bh2_med, bh2_work: Barnes-Hut (Algorithm 1, d = 2) at beta = 2, the paper's typical setting;
  its work is its far-field tests plus its terms;
- ratio: est_med / bh2_med (the paper's Table 1 has 2.4e-5 / 4.5e-4 = 0.053 at M = 2^20);
- bh_work_eq: Barnes-Hut's work at the estimator's median error, interpolated on log-log axes
  over beta in [0.5, 48] (Sec. 4.2, Fig. 4's rule); bh_work_eq / est_work < 1 means Barnes-Hut
  reaches the same median error with less work.

The last rows take the subdomains per query as the Barnes-Hut contribution nodes at beta_s (the
cover Sec. 3.3.1 names as future work); their work includes that walk's far-field tests.

This is a measurement script, not a test: it asserts nothing. The oracle is test infrastructure,
which is why the script lives beside the tests.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle as O  # noqa: E402
from paper_2506_02219_gb300 import workloads as W  # noqa: E402

BETAS = [0.5, 0.75, 1, 1.5, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48]
READINGS = [
    ("cell diagonal (built)", dict()),
    ("tight box, zero extent = cell", dict(box="tight")),
    ("tight box, literal (truncated)", dict(box="tight_literal")),
    ("cell, chains kept", dict(collapse=False)),
    ("cell, subdomains 2 generations down", dict(subdomain_generation=2)),
]
VARIANTS = [("roulette off", dict(rr=O.RR_OFF)), ("S = 4", dict(S=4))]


def case(n: int, seed: int = 11):
    P, w, _ = W.shape_union(n, seed, n_ellipsoids=1)
    return P, (w / w.sum()).astype(np.float32)


def query_sets(seed: int = 3, nq: int = 4096):
    rng = np.random.default_rng(seed)
    g = (np.arange(100) + 0.5) / 50.0 - 1.0
    grid = g[rng.integers(0, 100, (nq, 3))].astype(np.float32)
    rnd = rng.uniform(-1.0, 1.0, (nq, 3)).astype(np.float32)
    return {"grid": grid, "random": rnd}


def bh_work_at(t2, q, F, target):
    errs, work = [], []
    for b in BETAS:
        errs.append(np.median(np.abs(t2.bh(q, b) - F)))
        work.append(t2.bh_work(q, b).mean())
    le, lw = np.log(errs), np.log(work)
    o = np.argsort(le)
    return float(np.exp(np.interp(np.log(target), le[o], lw[o])))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 15)
    ap.add_argument("--seeds", type=int, default=8)
    args = ap.parse_args()
    P, w = case(args.n)
    t2 = O.Tree(P, w, d=2)
    qs = query_sets()
    Fs = {k: O.brute(P, w, q) for k, q in qs.items()}
    print(f"M = {args.n}, masses sum to 1; {args.seeds} seeds; Coulomb, softening 1e-3")
    hdr = ("reading", "queries", "est_med", "est_work", "bias", "bh2_med", "bh2_work", "ratio", "bh_work_eq/est_work")
    print(" | ".join(hdr))
    rows = [(name, opts, {}) for name, opts in READINGS] + [("cell, " + name, {}, v) for name, v in VARIANTS]
    for name, topts, eopts in rows:
        t = O.Tree(P, w, **topts)
        S = eopts.get("S", 1)
        rr = eopts.get("rr", O.RR_PAPER)
        for qname, q in qs.items():
            F = Fs[qname]
            errs, work = [], []
            for s in range(args.seeds):
                est, terms = t.replay(q, S=S, seed=1000 + s, rr=rr, return_terms=True)
                errs.append(np.abs(est - F))
                work.append(terms.mean())
            med, wk = float(np.median(np.concatenate(errs))), float(np.mean(work))
            mean, _ = t.enumerate(q[:256], rr=rr) if S == 1 else (F[:256], None)
            bias = float(np.median(np.abs(mean - F[:256])))
            bh2 = t2.bh(q, 2.0)
            bh2_med = float(np.median(np.abs(bh2 - F)))
            bh2_work = float(t2.bh_work(q, 2.0).mean())
            eq = bh_work_at(t2, q, F, med)
            print(f"{name} | {qname} | {med:.2e} | {wk:.0f} | {bias:.1e} | {bh2_med:.2e} | {bh2_work:.0f} | "
                  f"{med / bh2_med:.1f} | {eq / wk:.2f}", flush=True)
    t = O.Tree(P, w)
    for beta_s in (0.5, 1.0, 1.5, 2.0, 3.0):
        for qname, q in qs.items():
            F = Fs[qname]
            errs, work = [], []
            for s in range(args.seeds):
                est, wk = t.replay_cut(q, beta_s, seed=1000 + s)
                errs.append(np.abs(est - F))
                work.append(wk.mean())
            med, wk = float(np.median(np.concatenate(errs))), float(np.mean(work))
            mean, _ = t.enumerate_cut(q[:256], beta_s)
            bias = float(np.median(np.abs(mean - F[:256])))
            bh2_med = float(np.median(np.abs(t2.bh(q, 2.0) - F)))
            eq = bh_work_at(t2, q, F, med)
            print(f"cell, subdomains = Barnes-Hut cut at beta_s = {beta_s:g} | {qname} | {med:.2e} | {wk:.0f} | "
                  f"{bias:.1e} | {bh2_med:.2e} | {float(t2.bh_work(q, 2.0).mean()):.0f} | {med / bh2_med:.1f} | "
                  f"{eq / wk:.2f}", flush=True)


if __name__ == "__main__":
    main()
