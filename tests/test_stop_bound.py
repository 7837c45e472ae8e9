"""The certain-stop bound the estimator kernels use to skip decisions (host-side check of its
derivation, no GPU).

Before a path's child is drawn, the kernels test 4 u (d_T - B_T - slack) >= d_T (1 + 2^-10) in FP32
(u the roulette draw, d_T the FP32 distance from the query to the node's centre, B_T its cell
diagonal, slack = diam0 2^-19 + 2^-20 max |coordinate|) and, when it holds, drop the decision as a
stop. That is only valid if Eq. 5's exact test, u d_c < X with X = max(d_T, B_T) 4^-(l_c - l_T),
then fails for every child c. This test restates both tests in numpy FP32 with the kernels'
operation order and checks the implication at the smallest draw the bound accepts, for every
internal node of the oracle's trees (surface samples, a clustered cloud, and a tiny cloud far from
the origin where FP32 rounding of the coordinates is largest) at queries near and far.
"""
import numpy as np
import pytest

from paper_2506_02219_gb300 import workloads as W

f32 = np.float32


def _dist(p, q):
    d = (p - q).astype(f32)
    return np.sqrt((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]).astype(f32) + d[..., 2] * d[..., 2]).astype(f32)


def _slack(lo, side, diam0):
    c = f32(0)
    for a in range(3):
        c = max(c, abs(f32(lo[a])), abs(f32(f32(lo[a]) + f32(side))))
    return f32(f32(f32(diam0) * f32(2.0 ** -19)) + f32(c * f32(2.0 ** -20)))


def _smallest_stop_draw(dT, BT, slack):
    """Smallest u = k 2^-24 for which the FP32 certain-stop test holds (inf if none)."""
    g = f32(dT - f32(BT + slack))
    out = np.full(dT.shape, np.inf)
    ok = g > 0
    rhs = (dT * f32(1.0009765625)).astype(f32)
    gd = np.where(ok, g.astype(np.float64), 1.0)
    k = np.where(ok, np.ceil(rhs.astype(np.float64) / (4.0 * gd) * 2.0 ** 24) - 4, 2.0 ** 24)
    k = np.clip(k, 0, 2 ** 24)
    for _ in range(12):  # walk k up to the first value that passes the FP32 test
        u = (k * 2.0 ** -24).astype(f32)
        passed = ok & (k < 2 ** 24) & (f32(4) * u * np.where(ok, g, f32(0)) >= rhs)
        out = np.where(passed & np.isinf(out), u.astype(np.float64), out)
        k = k + 1
    return out


def _check(oracle_mod, pts, w, queries):
    t = oracle_mod.Tree(pts, w, d=4)
    e, m = t.export(), t.meta()
    com32 = e["com"].astype(f32)
    diam = [f32(np.ldexp(f32(m["diam0"]), -2 * lv)) for lv in range(12)]
    slack = _slack(m["lo"], m["side"], m["diam0"])
    internal = np.nonzero(e["nchild"] > 0)[0]
    checked = 0
    for q in queries.astype(f32):
        dT = _dist(com32[internal], q)
        BT = np.array([diam[lv] for lv in e["level"][internal]], f32)
        u = _smallest_stop_draw(dT, BT, slack)
        for i in np.nonzero(np.isfinite(u))[0]:
            v = internal[i]
            fc, nc = e["first_child"][v], e["nchild"][v]
            dc = _dist(com32[fc:fc + nc], q).astype(np.float64)
            shift = (e["level"][fc:fc + nc] - e["level"][v]).astype(np.int64)
            X = np.ldexp(np.float64(max(dT[i], BT[i])), -2 * shift)
            # Eq. 5 continues iff u d_c < X (exact in FP64 for a 24-bit u and FP32 d_c)
            assert np.all(u[i] * dc >= X), (v, u[i], dc.min(), X.max())
            checked += 1
    return checked


def test_bound_on_surface_samples(oracle_mod):
    P, wt, _ = W.shape_union(20000, 3, n_ellipsoids=4, n_boxes=2)
    rng = np.random.default_rng(1)
    q = np.concatenate([rng.uniform(-1.2, 1.2, (24, 3)), P[rng.integers(0, 20000, 8)] + 1e-3,
                        rng.uniform(-4, 4, (8, 3))])
    assert _check(oracle_mod, P, wt, q) > 10000


def test_bound_on_a_clustered_cloud(oracle_mod):
    rng = np.random.default_rng(2)
    P = np.concatenate([rng.random((3000, 3)), 0.3 + 1e-3 * rng.random((3000, 3))]).astype(np.float32)
    q = np.concatenate([rng.uniform(-0.2, 1.2, (24, 3)), P[:8] + 1e-5]).astype(np.float32)
    assert _check(oracle_mod, P, np.ones(6000, np.float32), q) > 1000


@pytest.mark.parametrize("offset,fires", [(1000.0, True), (-3.0e4, False)])
def test_bound_far_from_the_origin(oracle_mod, offset, fires):
    # a cloud 2e-3 across around x = offset. At 1000 FP32 rounding of coordinates is ~3e-2 of the
    # extent and the bound still fires far from the cloud; at -3e4 the coordinates' rounding step is
    # the whole extent, the slack exceeds every cell and the bound never fires (no decision skipped)
    rng = np.random.default_rng(3)
    P = (offset + 2e-3 * rng.random((4000, 3))).astype(np.float32)
    q = (offset + rng.uniform(-6e-3, 8e-3, (32, 3))).astype(np.float32)
    n = _check(oracle_mod, P, np.ones(4000, np.float32), q)
    assert (n > 100) if fires else (n == 0)
