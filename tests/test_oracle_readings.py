"""Pins of the oracle's alternative readings of the paper (oracle-only build options).

The CUDA path implements one reading of each point where the paper is loose. The oracle can
also build the others, so that what each does to the estimator can be measured:

- |B_a| as the tight axis-aligned box of the node's points (Sec. 3.1: "an axis-aligned bounding
  box containing all its points"), with zero-extent nodes taking their cell's diagonal: every
  Eq. 5 probability stays > 0, so the estimator stays unbiased (Appendix A).
- the literal tight box, |B| = 0 at a one-point node: beta~ is infinite there, Eq. 5 gives
  p = 0 and the swap above a one-point node is never taken. The estimator is truncated; a hand
  case fixes its mean exactly.
- single-child chains kept as nodes (their swaps are 0, so the mean is unchanged).
- subdomains taken g generations below the root (Sec. 3.3.1 allows any cover of the sources);
- subdomains taken per query as the Barnes-Hut contribution nodes at beta_s (the cover Sec. 3.3.1
  names as future work).

The last test keeps the measured finding these options serve: on a Table-1-like case (one
closed surface rescaled into [-1, 1]^3, masses summing to 1, the Coulomb kernel, grid and random
queries in the cube) the estimator at S = 1 has a larger median error than Barnes-Hut at
beta = 2 under every reading of |B_a| and of the chains.
"""
import numpy as np
import pytest

from paper_2506_02219_gb300 import workloads as W


def _problem(oracle_mod, n, seed, kind):
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3)).astype(np.float32)
    pts[: n // 3] = (0.2 + 0.05 * rng.random((n // 3, 3))).astype(np.float32)
    w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    nv = rng.normal(size=(n, 3))
    nv = (nv / np.linalg.norm(nv, axis=1, keepdims=True)).astype(np.float32)
    q = np.concatenate([rng.uniform(-0.3, 1.3, (6, 3)), pts[:2] + np.float32(1e-4), pts[2:3]]).astype(np.float32)
    k = dict(coulomb=oracle_mod.COULOMB, winding=oracle_mod.WINDING, smoothdist=oracle_mod.SMOOTHDIST)[kind]
    kw = dict(kind=k, softening=1e-3, alpha=30.0)
    normals = nv if kind == "winding" else None
    F = oracle_mod.brute(pts, w, q, normals=normals, **kw)
    return pts, w, normals, q, F, kw


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist"])
@pytest.mark.parametrize("opts", [dict(box="tight"), dict(collapse=False), dict(box="tight", collapse=False),
                                  dict(subdomain_generation=2), dict(subdomain_generation=3)],
                         ids=["tight", "no-collapse", "tight-no-collapse", "gen2", "gen3"])
@pytest.mark.parametrize("n,leaf", [(64, 1), (300, 1), (300, 4)])
def test_unbiased_readings_keep_the_theorem(oracle_mod, kind, opts, n, leaf):
    pts, w, normals, q, F, kw = _problem(oracle_mod, n, 7 + n, kind)
    t = oracle_mod.Tree(pts, w, normals, leaf_size=leaf, d=4, **opts)
    for rr in (oracle_mod.RR_PAPER, oracle_mod.RR_HALF):
        mean, var = t.enumerate(q, rr=rr, **kw)
        scale = np.maximum(np.abs(F), 1e-3 if kind == "winding" else 0.0)
        assert np.all(np.abs(mean - F) <= 1e-12 * scale + 1e-15), (mean - F) / scale
        assert np.all(var >= -1e-12 * scale * scale)


def test_literal_tight_box_truncates_at_one_point_nodes(oracle_mod):
    # A and B share a level-1 cell (subdomain {A, B}, whose children are the two points), C is
    # alone in another. With |B| = 0 at the one-point children, Eq. 5 gives p = 0: no path ever
    # leaves the subdomains, and the estimate is the sum of the two control variates.
    pts = np.array([[0.10, 0.10, 0.10], [0.12, 0.11, 0.10], [0.90, 0.90, 0.90]], np.float32)
    w = np.array([1.0, 2.0, 0.5], np.float32)
    q = np.array([[0.11, 0.30, 0.20], [0.5, 0.5, 0.5], [0.1, 0.1, 0.12]], np.float32)
    t = oracle_mod.Tree(pts, w, box="tight_literal")
    assert t.meta()["n_sub"] == 2
    p64, w64, q64 = pts.astype(np.float64), w.astype(np.float64), q.astype(np.float64)
    m_ab = w64[0] + w64[1]
    c_ab = (w64[0] * p64[0] + w64[1] * p64[1]) / m_ab
    eps2 = 1e-6
    cv = m_ab / np.sqrt(((c_ab - q64) ** 2).sum(1) + eps2) + w64[2] / np.sqrt(((p64[2] - q64) ** 2).sum(1) + eps2)
    mean, var = t.enumerate(q)
    np.testing.assert_allclose(mean, cv, rtol=1e-14)
    assert np.all(var <= 1e-28)
    for seed in range(5):
        np.testing.assert_allclose(t.replay(q, seed=seed), cv, rtol=1e-14)
    F = oracle_mod.brute(pts, w, q)
    assert np.all(np.abs(mean - F) > 1e-6 * F)  # truncated: biased
    # with the zero-extent rule the same swaps are reachable again and the mean is exact
    mean_t, _ = oracle_mod.Tree(pts, w, box="tight").enumerate(q)
    np.testing.assert_allclose(mean_t, F, rtol=1e-12)


def test_tight_box_changes_the_far_field_test(oracle_mod):
    # Two close points and one far point, d = 2. Root cube: corner 0.2, edge 0.75. The pair's x
    # cells (0 and floor(0.01 / 0.75 * 2^20) = 13981 < 2^14) first differ in bit 13, so the pair
    # is one node at level 6 (cell diagonal 0.75 sqrt(3) / 64 = 0.0203) whose children are the
    # points. Its tight box diagonal is |A - B| = 0.01. At 0.03 from the pair's centre,
    # beta~ = 1.48 under the cell reading (Algorithm 1 opens the pair: exact) and 3 under the tight
    # reading (it accepts the pair as one term at beta = 2).
    pts = np.array([[0.20, 0.20, 0.20], [0.21, 0.20, 0.20], [0.95, 0.95, 0.95]], np.float32)
    w = np.array([1.0, 1.0, 1.0], np.float32)
    q = np.array([[0.205, 0.23, 0.20]], np.float32)
    p64 = pts.astype(np.float64)
    com = 0.5 * (p64[0] + p64[1])
    mono = 2.0 / np.sqrt(((com - q[0]) ** 2).sum() + 1e-6) + 1.0 / np.sqrt(((p64[2] - q[0]) ** 2).sum() + 1e-6)
    F = oracle_mod.brute(pts, w, q)
    np.testing.assert_allclose(oracle_mod.Tree(pts, w, d=2, box="tight").bh(q, 2.0), [mono], rtol=1e-14)
    np.testing.assert_allclose(oracle_mod.Tree(pts, w, d=2).bh(q, 2.0), F, rtol=1e-14)
    # at 0.015 the tight reading's beta~ is 1.5: the pair is opened (a half diagonal would accept it)
    q2 = np.array([[0.205, 0.215, 0.20]], np.float32)
    np.testing.assert_allclose(oracle_mod.Tree(pts, w, d=2, box="tight").bh(q2, 2.0), oracle_mod.brute(pts, w, q2),
                               rtol=1e-14)


def test_chains_kept_as_nodes(oracle_mod):
    # two points that share their level-1 and level-2 cells and split at level 3
    pts = np.array([[0.001, 0.001, 0.001], [0.02, 0.001, 0.001], [0.999, 0.999, 0.999]], np.float32)
    w = np.ones(3, np.float32)
    e1 = oracle_mod.Tree(pts, w).export()
    e0 = oracle_mod.Tree(pts, w, collapse=False).export()
    # collapsed: root, {A, B} at the level where they split, C, A, B
    assert e1["nchild"].tolist() == [2, 2, 0, 0, 0] and e1["level"].tolist() == [0, 2, 1, 3, 3]
    # kept: root, {A, B} at level 1, C, {A, B} at level 2, A, B
    assert e0["nchild"].tolist() == [2, 1, 0, 2, 0, 0] and e0["level"].tolist() == [0, 1, 1, 2, 3, 3]


def _generations(e):
    N = e["nchild"].shape[0]
    gen = np.zeros(N, np.int64)
    for v in range(N):
        fc, nc = e["first_child"][v], e["nchild"][v]
        if nc:
            gen[fc:fc + nc] = gen[v] + 1
    return gen


@pytest.mark.parametrize("g", [1, 2, 3])
def test_subdomain_generation_cover(oracle_mod, g):
    pts, w, normals, q, F, kw = _problem(oracle_mod, 300, 4, "coulomb")
    t = oracle_mod.Tree(pts, w, subdomain_generation=g)
    e = t.export()
    gen = _generations(e)
    subs = np.nonzero((gen == g) | ((gen < g) & (gen > 0) & (e["nchild"] == 0)))[0]
    assert t.meta()["n_sub"] == subs.size and t.meta()["first_sub"] == subs[0]
    # the subdomains partition the points (Sec. 3.3.1: they must cover every source once)
    cover = np.zeros(300, np.int64)
    for v in subs:
        cover[e["begin"][v]:e["end"][v]] += 1
    assert np.all(cover == 1)


def test_leaf_subdomains_give_the_exact_sum(oracle_mod):
    pts, w, normals, q, F, kw = _problem(oracle_mod, 200, 2, "coulomb")
    t = oracle_mod.Tree(pts, w, subdomain_generation=40)
    assert t.meta()["n_sub"] == 200
    np.testing.assert_allclose(t.replay(q, seed=1), F, rtol=1e-13)


def test_estimator_loses_to_barnes_hut_on_a_table1_like_case(oracle_mod):
    P, wt, _ = W.shape_union(4096, 11, n_ellipsoids=1)
    wt = (wt / wt.sum()).astype(np.float32)
    rng = np.random.default_rng(3)
    g = (np.arange(100) + 0.5) / 50.0 - 1.0
    grid = g[rng.integers(0, 100, (256, 3))]
    q = np.concatenate([grid, rng.uniform(-1, 1, (256, 3))]).astype(np.float32)
    F = oracle_mod.brute(P, wt, q)
    e_bh = np.median(np.abs(oracle_mod.Tree(P, wt, d=2).bh(q, 2.0) - F))
    for opts in (dict(), dict(box="tight"), dict(box="tight_literal"), dict(collapse=False)):
        t = oracle_mod.Tree(P, wt, **opts)
        e_est = np.median(np.abs(np.concatenate([t.replay(q, seed=s) for s in range(8)]) - np.tile(F, 8)))
        assert e_est > 5.0 * e_bh, (opts, e_est, e_bh)


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist"])
@pytest.mark.parametrize("beta_s", [0.5, 1.0, 2.0])
def test_barnes_hut_cut_subdomains_keep_the_theorem(oracle_mod, kind, beta_s):
    pts, w, normals, q, F, kw = _problem(oracle_mod, 300, 31, kind)
    t = oracle_mod.Tree(pts, w, normals)
    mean, var = t.enumerate_cut(q, beta_s, **kw)
    scale = np.maximum(np.abs(F), 1e-3 if kind == "winding" else 0.0)
    assert np.all(np.abs(mean - F) <= 1e-12 * scale + 1e-15), (mean - F) / scale
    assert np.all(var >= -1e-12 * scale * scale)


def test_barnes_hut_cut_limits(oracle_mod):
    pts, w, normals, q, F, kw = _problem(oracle_mod, 200, 8, "coulomb")
    t = oracle_mod.Tree(pts, w)
    # beta_s = inf: the cut is every leaf (here every source point), so the estimate is the exact sum
    est, work = t.replay_cut(q, float("inf"), seed=3)
    np.testing.assert_allclose(est, F, rtol=1e-13)
    assert np.all(work == t.n_nodes)  # every node tested once, no swap
    # beta_s = 0: the root alone is the cut; unbiased, with variance
    mean, var = t.enumerate_cut(q, 0.0)
    np.testing.assert_allclose(mean, F, rtol=1e-12)
    assert np.all(var > 0)
    # the replay samples that distribution: the mean of many seeds approaches the exact sum
    est = np.mean([t.replay_cut(q, 1.0, seed=s)[0] for s in range(400)], axis=0)
    m1, v1 = t.enumerate_cut(q, 1.0)
    assert np.all(np.abs(est - m1) <= 5 * np.sqrt(v1 / 400) + 1e-12 * np.abs(m1))
