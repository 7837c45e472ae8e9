"""Pins of the oracle's estimator (Sec. 3.3, Eq. 5-7, Algorithm 2) and Barnes-Hut (Algorithm 1).

- The theorem (Sec. 3.3, proof in Appendix A): E[F_1(q)] = F(q). The oracle enumerates every
  outcome of the path sampler on small trees; its mean must equal the brute-force sum to 1e-12,
  for every kernel, both path-index distributions and every Russian-roulette rule. A dropped
  weight, a wrong p(I in T) or p(K >= k), or a sign error in the swap breaks this.
- Affine kernels: sum_c m_c p_c = m_T p_T makes every swap (Eq. 6) vanish, so the estimator is
  exact with zero variance.
- A tree whose subdomains are all source points is summed exactly (every path stops at once).
- The replay (Philox-driven) is a sample of the enumerated distribution: over many seeds its mean
  and variance match the enumerated mean and variance.
- Barnes-Hut with beta = inf visits every leaf (exact); with beta = 0 it returns the root's
  aggregate term M f(p_com, q).
"""
import math

import numpy as np
import pytest

KINDS = ["coulomb", "winding", "smoothdist", "affine"]


def _setup(oracle_mod, n, seed, kind, leaf_size=1):
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3)).astype(np.float32)
    if n > 4:  # a clustered part so that some subtrees are deep
        pts[: n // 3] = (0.2 + 0.05 * rng.random((n // 3, 3))).astype(np.float32)
    w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    nv = rng.normal(size=(n, 3))
    nv = (nv / np.linalg.norm(nv, axis=1, keepdims=True)).astype(np.float32)
    q = np.concatenate([rng.uniform(-0.3, 1.3, (6, 3)), pts[:2] + np.float32(1e-4), pts[2:3]]).astype(np.float32)
    k = dict(coulomb=oracle_mod.COULOMB, winding=oracle_mod.WINDING, smoothdist=oracle_mod.SMOOTHDIST,
             affine=oracle_mod.AFFINE)[kind]
    kw = dict(kind=k, softening=1e-3, alpha=30.0, affine=(0.4, -0.3, 0.8))
    t = oracle_mod.Tree(pts, w, nv if kind == "winding" else None, leaf_size=leaf_size, d=4)
    F = oracle_mod.brute(pts, w, q, normals=nv if kind == "winding" else None, **kw)
    return t, q, F, kw


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("sampling", [0, 1])
@pytest.mark.parametrize("rr", [0, 1, 2])
@pytest.mark.parametrize("n,leaf", [(2, 1), (9, 1), (64, 1), (300, 1), (300, 4)])
def test_enumeration_mean_equals_brute_force(oracle_mod, kind, sampling, rr, n, leaf):
    t, q, F, kw = _setup(oracle_mod, n, 100 + n, kind, leaf)
    mean, var = t.enumerate(q, sampling=sampling, rr=rr, **kw)
    scale = np.maximum(np.abs(F), 1e-3 if kind == "winding" else 0.0)
    assert np.all(np.abs(mean - F) <= 1e-12 * scale + 1e-15), (mean - F) / scale
    assert np.all(var >= -1e-12 * scale * scale)


def test_affine_kernel_has_zero_variance(oracle_mod):
    t, q, F, kw = _setup(oracle_mod, 300, 5, "affine")
    mean, var = t.enumerate(q, **kw)
    assert np.all(var <= 1e-22 * F * F)
    for seed in (0, 1, 12345):
        est = t.replay(q, S=1, seed=seed, **kw)
        np.testing.assert_allclose(est, F, rtol=1e-12)


def test_subdomains_that_are_points_give_the_exact_sum(oracle_mod):
    # 4x4x4 cell centres: each point alone in its level-1 cell, so every subdomain is a point
    g = (np.arange(4) + 0.5) / 4
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    w = np.random.default_rng(0).uniform(0.5, 1.5, 64).astype(np.float32)
    t = oracle_mod.Tree(pts, w, d=4)
    assert t.meta()["n_sub"] == 64 and t.export()["nchild"][1:].max() == 0
    q = np.random.default_rng(1).random((10, 3)).astype(np.float32)
    F = oracle_mod.brute(pts, w, q)
    np.testing.assert_allclose(t.replay(q, seed=3), F, rtol=1e-14)


@pytest.mark.parametrize("sampling,rr", [(0, 0), (1, 0), (0, 2)])
def test_replay_samples_the_enumerated_distribution(oracle_mod, sampling, rr):
    t, q, F, kw = _setup(oracle_mod, 40, 9, "coulomb")
    mean, var = t.enumerate(q, sampling=sampling, rr=rr, **kw)
    n_seeds = 3000
    est = np.stack([t.replay(q, S=1, seed=s, sampling=sampling, rr=rr, **kw) for s in range(n_seeds)])
    smean = est.mean(0)
    svar = est.var(0, ddof=1)
    sigma = np.sqrt(var / n_seeds)
    nz = var > 1e-12 * F * F
    assert np.all(np.abs(smean - mean)[nz] <= 4.5 * sigma[nz])
    ratio = svar[nz] / var[nz]
    assert np.all((ratio > 0.75) & (ratio < 1.3)), ratio


def test_samples_per_subdomain_divide_the_variance(oracle_mod):
    t, q, F, kw = _setup(oracle_mod, 40, 21, "coulomb")
    _, var = t.enumerate(q[:4], **kw)
    est = np.stack([t.replay(q[:4], S=4, seed=s, **kw) for s in range(2000)])
    ratio = est.var(0, ddof=1) / (var / 4)
    assert np.all((ratio > 0.75) & (ratio < 1.3)), ratio


def test_replay_is_deterministic_per_seed(oracle_mod):
    t, q, F, kw = _setup(oracle_mod, 300, 8, "coulomb")
    a = t.replay(q, seed=77, **kw)
    np.testing.assert_array_equal(a, t.replay(q, seed=77, **kw))
    assert np.any(a != t.replay(q, seed=78, **kw))


def test_rr_off_has_no_more_variance_in_aggregate(oracle_mod):
    t, q, F, kw = _setup(oracle_mod, 300, 12, "coulomb")
    _, v_rr = t.enumerate(q, rr=0, **kw)
    _, v_off = t.enumerate(q, rr=1, **kw)
    assert v_off.sum() <= v_rr.sum()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("d", [4, 2])
def test_barnes_hut_limits(oracle_mod, kind, d):
    t, q, F, kw = _setup(oracle_mod, 300, 31, kind)
    t = oracle_mod.Tree(t.points, t.weights, t.normals, leaf_size=1, d=d)
    exact = t.bh(q, np.inf, **kw)
    scale = np.maximum(np.abs(F), 1e-3 if kind == "winding" else 0.0)
    assert np.all(np.abs(exact - F) <= 1e-12 * scale + 1e-15)
    # beta = 0: only the root, i.e. the total mass at the centre of mass
    root = t.bh(q, 0.0, **kw)
    m = t.weights.astype(np.float64)
    com = (m[:, None] * t.points.astype(np.float64)).sum(0) / m.sum()
    d = np.linalg.norm(com[None] - q.astype(np.float64), axis=1)
    if kind == "coulomb":
        ref = m.sum() / np.sqrt(d * d + 1e-6)
    elif kind == "smoothdist":
        ref = m.sum() * np.exp(-30.0 * d)
    elif kind == "affine":
        ref = m.sum() * (1.0 + (com[None] - q.astype(np.float64)) @ np.array([0.4, -0.3, 0.8]))
    else:
        dip = (m[:, None] * t.normals.astype(np.float64)).sum(0)
        ref = ((com[None] - q.astype(np.float64)) @ dip) / (4 * math.pi * d ** 3)
    np.testing.assert_allclose(root, ref, rtol=1e-12)


def test_barnes_hut_error_shrinks_with_beta(oracle_mod):
    rng = np.random.default_rng(2)
    pts = rng.random((4000, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 4000).astype(np.float32)
    q = rng.random((200, 3)).astype(np.float32)
    F = oracle_mod.brute(pts, w, q)
    t = oracle_mod.Tree(pts, w, d=2)
    errs = [np.mean(np.abs(t.bh(q, b) - F) / F) for b in (1.0, 2.0, 4.0, 8.0)]
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[1] < 1e-2


def test_abs_sum_bounds_the_estimate(oracle_mod):
    """The replay's abs_sum (sum of |terms| the estimate adds) is >= |estimate|, equals the
    estimate when every term is positive (subdomains that are points, Coulomb), and scales with S."""
    t, q, F, kw = _setup(oracle_mod, 300, 14, "smoothdist")
    est, A = t.replay(q, S=2, seed=4, return_abs_sum=True, **kw)
    assert np.all(A >= np.abs(est) * (1 - 1e-12))
    g = (np.arange(4) + 0.5) / 4
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    w = np.full(64, 0.7, np.float32)
    tp = oracle_mod.Tree(pts, w, d=4)
    est, A = tp.replay(q, seed=1, return_abs_sum=True)
    np.testing.assert_allclose(A, est, rtol=1e-14)



def test_fp32_record_sensitivity_scale(oracle_mod):
    """abs_mode=1 scales each winding term by |N| (r + 4 |p|) / (4 pi r^3) >= |term|, so its sum is
    at least the plain abs_sum; the other kernels ignore the mode. The scale bounds what rounding
    a node's record (centre of mass and dipole) to FP32 does to its term: at queries on the
    sources of a surface-sample tree, every internal node's term moves by at most 2^-24 times it."""
    t, q, F, kw = _setup(oracle_mod, 300, 14, "winding")
    _, A0 = t.replay(q, S=2, seed=4, return_abs_sum=True, **kw)
    _, A1 = t.replay(q, S=2, seed=4, return_abs_sum=True, abs_mode=1, **kw)
    assert np.all(A1 >= A0 * (1 - 1e-12)) and np.any(A1 > 2 * A0)
    for kind in ("coulomb", "smoothdist"):
        t2, q2, _, kw2 = _setup(oracle_mod, 300, 14, kind)
        _, B0 = t2.replay(q2, S=2, seed=4, return_abs_sum=True, **kw2)
        _, B1 = t2.replay(q2, S=2, seed=4, return_abs_sum=True, abs_mode=1, **kw2)
        np.testing.assert_array_equal(B0, B1)
    from paper_2506_02219_gb300 import workloads as W
    pts, w, nrm = W.shape_union(3000, 5, n_ellipsoids=2, n_boxes=1)
    e = oracle_mod.Tree(pts, w, nrm, leaf_size=1, d=4).export()
    inner = e["nchild"] > 0
    com, dip = e["com"][inner], e["dip"][inner]
    com32 = com.astype(np.float32).astype(np.float64)
    dip32 = dip.astype(np.float32).astype(np.float64)
    for qq in pts[::25].astype(np.float64):
        d, d32 = com - qq, com32 - qq
        r, r32 = np.linalg.norm(d, axis=1), np.linalg.norm(d32, axis=1)
        t64 = (d * dip).sum(1) / (4 * np.pi * r ** 3)
        t32 = (d32 * dip32).sum(1) / (4 * np.pi * r32 ** 3)
        scale = np.linalg.norm(dip, axis=1) * (r + 4 * np.linalg.norm(com, axis=1)) / (4 * np.pi * r ** 3)
        assert np.all(np.abs(t32 - t64) <= 2.0 ** -24 * scale), np.max(np.abs(t32 - t64) / (2.0 ** -24 * scale))
