"""The adjoint (sbh_eval_grad) on the GPU against the oracle.

- Parity with the oracle's gradient replay (same paths and weights, FP32 decisions on both
  sides): |g_gpu - g_oracle| <= 1e-4 * A_g on >= 99.9% of queries, A_g the sum of |gradient terms|,
  for the warp-task kernel and the one-thread-per-query kernel.
- Unbiasedness: averaged over seeds, the GPU gradient of the sum lies within 3 sigma of the
  FP64 brute-force gradient of Eq. 1.
- Finite differences: with the roulette off (p = 1) and mass-proportional picks no decision and no
  weight depends on q, so central differences (h = 1e-4) of the GPU's own estimate are the
  derivative the adjoint computes. (With Eq. 5 the weights 1/p_rr vary smoothly with q; the adjoint
  holds them fixed, which is what makes it unbiased, and the oracle pins it against frozen-path
  finite differences.) For the smooth distance, at many samples the adjoint of d = -log(F)/alpha
  approaches the FP64 brute-force gradient.
- torch.autograd: StochasticSum's backward is the adjoint.
- The GPU brute-force gradient (the bench's error reference for the adjoint) against the oracle's
  FP64 brute-force value and gradient.
"""
import numpy as np
import pytest

from gpu_util import dev, gpu_kwargs, oracle_kwargs

pytestmark = pytest.mark.gpu


def _inputs(kind, n, nq, seed):
    from paper_2506_02219_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    if kind in ("winding", "smoothdist"):
        pts, w, nrm = W.shape_union(n, seed, n_ellipsoids=5, n_boxes=1)
        if kind == "smoothdist":
            w, nrm = np.ones_like(w), None
        q = rng.uniform(-1.05, 1.05, (nq, 3)).astype(np.float32)
    else:
        pts = rng.random((n, 3)).astype(np.float32)
        w = rng.uniform(0.5, 1.5, n).astype(np.float32)
        nrm = None
        q = rng.uniform(-0.1, 1.1, (nq, 3)).astype(np.float32)
    return pts, w, nrm, q


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist", "affine"])
@pytest.mark.parametrize("S,schedule", [(1, 0), (2, 0), (1, 1), (2, 1)])
def test_adjoint_matches_oracle(sbh, oracle_mod, kind, S, schedule):
    pts, w, nrm, q = _inputs(kind, 10000, 2001, 61 + S)
    alpha = 30.0
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    o = sbh.EvalOpts()
    o.raw_sum = 1  # smooth distance: compare the sum and its gradient
    o.schedule = schedule  # 0: warp-task kernel, 1: one thread per query
    val, g = sbh.sbh_eval_grad(t, dev(q), samples_per_subdomain=S, seed=5, opts=o, **gpu_kwargs(kind, alpha=alpha))
    val, g = val.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    ot = oracle_mod.Tree(pts, w, nrm, leaf_size=1, d=4)
    kw = oracle_kwargs(oracle_mod, kind, alpha=alpha)
    ov, og, A = ot.replay_grad(q, S=S, seed=5, **kw)
    err = np.abs(g - og).max(1) / A
    assert np.mean(err <= 1e-4) >= 0.999, np.sort(err)[-5:]
    _, Av = ot.replay(q, S=S, seed=5, return_abs_sum=True, **kw)
    errv = np.abs(val - ov) / np.maximum(Av, 1.0 if kind == "winding" else 0.0)
    assert np.mean(errv <= 1e-4) >= 0.999


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist"])
def test_adjoint_is_unbiased(sbh, oracle_mod, kind):
    pts, w, nrm, q = _inputs(kind, 400, 10, 71)
    alpha = 30.0
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    o = sbh.EvalOpts()
    o.raw_sum = 1
    Q = dev(q)
    K = 2000
    gs = np.stack([sbh.sbh_eval_grad(t, Q, seed=s, opts=o, **gpu_kwargs(kind, alpha=alpha))[1].cpu().numpy()
                   for s in range(K)]).astype(np.float64)
    G = oracle_mod.brute_grad(pts, w, q, normals=nrm, **oracle_kwargs(oracle_mod, kind, alpha=alpha))
    se = gs.std(0, ddof=1) / np.sqrt(K)
    z = np.abs(gs.mean(0) - G) / np.maximum(se, 1e-7 * np.abs(G).max(1, keepdims=True) + 1e-30)
    assert np.mean(z <= 3.0) >= 0.95 and np.all(z <= 5.0), np.sort(z.ravel())[-6:]


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist"])
@pytest.mark.parametrize("schedule", [0, 1])
def test_adjoint_matches_finite_differences_without_roulette(sbh, oracle_mod, kind, schedule):
    pts, w, nrm, q = _inputs(kind, 20000, 81, 512)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    kw = gpu_kwargs(kind, alpha=200.0)
    o = sbh.EvalOpts()
    o.rr = 1
    o.schedule = schedule
    d0, g = sbh.sbh_eval_grad(t, dev(q), seed=9, opts=o, **kw)
    d0, g = d0.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    ok = np.isfinite(d0)
    h = 1e-4
    fd = np.zeros_like(g)
    for a in range(3):
        e = np.zeros(3, np.float32)
        e[a] = h
        dp = sbh.sbh_eval(t, dev(q + e), seed=9, opts=o, **kw).cpu().numpy().astype(np.float64)
        dm = sbh.sbh_eval(t, dev(q - e), seed=9, opts=o, **kw).cpu().numpy().astype(np.float64)
        fin = np.isfinite(dp) & np.isfinite(dm)  # a smooth distance is +inf where its estimate is <= 0
        fd[:, a] = np.where(fin, (np.where(fin, dp, 0.0) - np.where(fin, dm, 0.0)) / (2 * h), np.nan)
        ok &= fin
    # FP32 estimates: the difference quotient carries ~1e-7 |F| / h of rounding
    scale = np.abs(g).max(1) + 1e-3 * np.abs(d0) / h
    rel = np.abs(fd - g).max(1)[ok] / scale[ok]
    assert np.median(rel) < 5e-3 and np.mean(rel < 5e-2) > 0.95, (np.median(rel), np.mean(rel < 5e-2))


def test_smooth_distance_gradient_approaches_exact(sbh, oracle_mod):
    from paper_2506_02219_gb300 import workloads as W
    pts, w, _ = W.shape_union(30000, 81, n_ellipsoids=6, n_boxes=2)
    w = np.ones_like(w)
    q = np.random.default_rng(3).uniform(-1.0, 1.0, (128, 3)).astype(np.float32)
    t = sbh.sbh_build(dev(pts), dev(w))
    d64, g64 = sbh.sbh_eval_grad(t, dev(q), samples_per_subdomain=64, seed=1, **gpu_kwargs("smoothdist"))
    F = oracle_mod.brute(pts, w, q, kind=oracle_mod.SMOOTHDIST, alpha=200.0)
    GF = oracle_mod.brute_grad(pts, w, q, kind=oracle_mod.SMOOTHDIST, alpha=200.0)
    gd = -GF / (200.0 * F[:, None])  # gradient of -log(F)/alpha
    e = np.abs(g64.cpu().numpy() - gd).max(1) / np.abs(gd).max(1)
    fin = np.isfinite(e)  # NaN where the estimate of F is <= 0: no distance, no gradient
    assert fin.mean() >= 0.9 and np.median(e[fin]) < 0.1, (fin.mean(), np.median(e[fin]))


def test_autograd_backward_is_the_adjoint(sbh):
    import torch
    pts, w, nrm, q = _inputs("coulomb", 5000, 300, 91)
    t = sbh.sbh_build(dev(pts), dev(w))
    Q = dev(q).requires_grad_(True)
    out = sbh.StochasticSum(Q, t, "coulomb", 1, 17)
    (out * torch.arange(1, 301, device="cuda", dtype=torch.float32)).sum().backward()
    _, g = sbh.sbh_eval_grad(t, dev(q), "coulomb", 1, 17)
    ref = g * torch.arange(1, 301, device="cuda", dtype=torch.float32)[:, None]
    torch.testing.assert_close(Q.grad, ref)
    val = sbh.sbh_eval(t, dev(q), "coulomb", 1, 17)
    torch.testing.assert_close(out.detach(), val, rtol=1e-5, atol=0)


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist", "affine"])
def test_brute_gradient_matches_oracle(sbh, oracle_mod, kind):
    """sbh_eval_brute_grad against the oracle's FP64 brute-force value and gradient: FP32 tile
    partials added in FP64 leave errors near FP32 rounding of one tile (1e-5 of the scale)."""
    pts, w, nrm, q = _inputs(kind, 5000, 700, 61)
    kw = oracle_kwargs(oracle_mod, kind, alpha=30.0)
    F = oracle_mod.brute(pts, w, q, normals=nrm, **kw)
    G = oracle_mod.brute_grad(pts, w, q, normals=nrm, **kw)
    out, grad = sbh.sbh_eval_brute_grad(dev(pts), dev(w), dev(q), normals=dev(nrm), **gpu_kwargs(kind, alpha=30.0))
    out, grad = out.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64)
    if kind == "smoothdist":  # distance and its gradient -grad F / (alpha F)
        F, G = -np.log(F) / 30.0, -G / (30.0 * F[:, None])
    scale = np.abs(G).max()
    assert np.all(np.abs(grad - G) <= 1e-5 * scale + 1e-5 * np.abs(G)), np.abs(grad - G).max() / scale
    np.testing.assert_allclose(out, F, rtol=1e-5, atol=1e-6 * np.abs(F).max())
