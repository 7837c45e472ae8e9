"""The learned child proposal on the GPU (a project extension of Sec. 3.3's path sampling).

- Scores of the FP16-weight inference network against the oracle's FP64 network evaluated on the
  same FP16-rounded weights (FP32 accumulation: within 1e-4 of the scale of the terms).
- Training loss and gradient (FP32 master weights) against the oracle's FP64 loss and gradient.
- The training set (features and |exact child residual| targets) against the oracle's features and
  brute-force residuals.
- Unbiasedness: seed-averaged learned estimates within 4 sigma of the exact sum, sigma from the
  oracle's enumerated variance of the one-sample learned estimator.
- Training lowers the loss, and the trained proposal has lower variance than the mass-proportional
  pick on held-out queries.
"""
import numpy as np
import pytest

from gpu_util import dev, gpu_kwargs, oracle_kwargs

pytestmark = pytest.mark.gpu


def _rand_weights(oracle_mod, seed, scale=0.3):
    return np.random.default_rng(seed).normal(scale=scale, size=oracle_mod.MLP_NPARAM).astype(np.float32)


def test_scores_match_oracle(sbh, oracle_mod):
    w = _rand_weights(oracle_mod, 1)
    net = sbh.sbh_mlp_create(0)
    sbh.sbh_mlp_set_weights(net, w)
    x = np.random.default_rng(2).normal(size=(5000, 6)).astype(np.float32)
    g = sbh.sbh_mlp_scores(net, dev(x)).cpu().numpy().astype(np.float64)
    wh = w.astype(np.float16).astype(np.float64)
    ref = oracle_mod.mlp_forward(wh, x.astype(np.float64))
    # scale: the same network with |weights| and |inputs| bounds every partial sum
    a = np.abs(wh)
    scale = oracle_mod.mlp_forward(a, np.abs(x).astype(np.float64))
    assert np.all(np.abs(g - ref) <= 1e-4 * scale + 1e-6), np.max(np.abs(g - ref) / scale)


@pytest.mark.parametrize("sizes", [[2, 5, 17, 64], [3] * 200 + [64] * 40])
def test_loss_grad_matches_oracle(sbh, oracle_mod, sizes):
    import torch
    rng = np.random.default_rng(len(sizes))
    w = _rand_weights(oracle_mod, 3)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = rng.normal(size=(off[-1], 6)).astype(np.float32)
    t = rng.random(off[-1]).astype(np.float32)
    t[off[1]:off[2]] = 0.0  # one set with all-zero targets (uniform)
    net = sbh.sbh_mlp_create(0)
    sbh.sbh_mlp_set_weights(net, w)
    loss, grad = sbh.sbh_mlp_loss_grad(net, dev(x), dev(t), torch.from_numpy(off).cuda())
    ref_loss, ref_g = oracle_mod.mlp_loss_grad(w.astype(np.float64), x.astype(np.float64), t.astype(np.float64), off)
    assert abs(float(loss.item()) - ref_loss) <= 1e-4 * abs(ref_loss)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * np.max(np.abs(ref_g)), np.max(np.abs(g - ref_g)) / np.max(np.abs(ref_g))


def test_weights_round_trip(sbh, oracle_mod):
    w = _rand_weights(oracle_mod, 4)
    net = sbh.sbh_mlp_create(7)
    sbh.sbh_mlp_set_weights(net, w)
    back, step = sbh.sbh_mlp_get_weights(net)
    assert step == 0 and np.array_equal(back, w)
    a, _ = sbh.sbh_mlp_get_weights(sbh.sbh_mlp_create(7))
    b, _ = sbh.sbh_mlp_get_weights(sbh.sbh_mlp_create(7))
    assert np.array_equal(a, b) and np.all(np.isfinite(a)) and np.any(a != 0)


def _shapes(n, nq, seed, kind):
    from paper_2506_02219_gb300 import workloads as W
    pts, w, nrm = W.shape_union(n, seed, n_ellipsoids=6, n_boxes=2)
    if kind != "winding":
        nrm = None
    if kind == "smoothdist":
        w = np.ones_like(w)
    q = np.random.default_rng(seed + 1).uniform(-1.05, 1.05, (nq, 3)).astype(np.float32)
    return pts, w, nrm, q


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist", "affine"])
def test_learned_seed_mean_within_four_sigma(sbh, oracle_mod, kind):
    pts, w, nrm, q = _shapes(400, 10, 41, kind)
    kw = oracle_kwargs(oracle_mod, kind, alpha=30.0)
    wt = _rand_weights(oracle_mod, 5, 0.5)
    ot = oracle_mod.Tree(pts, w, nrm, leaf_size=1, d=4)
    F = oracle_mod.brute(pts, w, q, normals=nrm, **kw)
    _, var = ot.enumerate_learned(q, wt.astype(np.float16).astype(np.float64), 0.1, **kw)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    net = sbh.sbh_mlp_create(0)
    sbh.sbh_mlp_set_weights(net, wt)
    o = sbh.EvalOpts()
    o.raw_sum = 1
    Q = dev(q)
    K = 2000
    est = np.stack([sbh.sbh_eval_learned(t, net, Q, seed=s, opts=o, **gpu_kwargs(kind, alpha=30.0)).cpu().numpy()
                    for s in range(K)]).astype(np.float64)
    sigma = np.sqrt(np.maximum(var, 0.0) / K)
    dev_ = np.abs(est.mean(0) - F)
    assert np.all(dev_ <= 4 * sigma + 2e-6 * np.abs(F) + 1e-7), dev_ / np.maximum(sigma, 1e-30)
    if kind == "affine":  # zero variance under any proposal
        assert np.all(np.abs(est - F) <= 1e-4 * np.abs(F))


def test_training_set_matches_oracle_residuals(sbh, oracle_mod):
    """The first Adam step's loss equals the oracle's loss on the oracle's features and residual
    targets for the same decision sets (the subdomains' children), at the same weights."""
    kind = "winding"
    pts, w, nrm, q = _shapes(3000, 16, 43, kind)
    kw = oracle_kwargs(oracle_mod, kind)
    ot = oracle_mod.Tree(pts, w, nrm, leaf_size=1, d=4)
    e = ot.export()
    wt = _rand_weights(oracle_mod, 6)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    net = sbh.sbh_mlp_create(0)
    sbh.sbh_mlp_set_weights(net, wt)
    losses = sbh.sbh_mlp_train(net, t, dev(q), kernel=kind, steps=1, lr=1e-3)
    # oracle side: the same sets, targets = |exact sum over the child's points - its own term|
    m = ot.meta()
    subs = [a for a in range(m["first_sub"], m["first_sub"] + m["n_sub"]) if 2 <= e["nchild"][a] <= 64]
    feats, targ, off = [], [], [0]
    order = e["perm"]
    spts, sw, snrm = pts[order], w[order], nrm[order]
    for j in range(q.shape[0]):
        for a in subs:
            x = ot.child_features(a, q[j], True)
            f = int(e["first_child"][a])
            for c in range(int(e["nchild"][a])):
                b, en = int(e["begin"][f + c]), int(e["end"][f + c])
                exact = oracle_mod.brute(spts[b:en], sw[b:en], q[j:j + 1], normals=snrm[b:en], **kw)[0]
                # the child's own term at its FP32 centre of mass: its dipole sum(m n) for winding numbers
                own = oracle_mod.brute(e["com"][f + c:f + c + 1].astype(np.float32), np.ones(1, np.float32),
                                       q[j:j + 1], normals=e["dip"][f + c:f + c + 1].astype(np.float32), **kw)[0]
                targ.append(abs(exact - own))
            feats.append(x)
            off.append(off[-1] + x.shape[0])
    ref_loss, _ = oracle_mod.mlp_loss_grad(wt.astype(np.float64), np.concatenate(feats), np.array(targ), off)
    assert abs(float(losses[0]) - ref_loss) <= 2e-4 * abs(ref_loss), (losses[0], ref_loss)


def _variance(sbh, t, net, Q, kind, rr, K):
    o = sbh.EvalOpts()
    o.rr = rr
    o.raw_sum = 1
    f = (lambda s: sbh.sbh_eval_learned(t, net, Q, seed=s, opts=o, **gpu_kwargs(kind))) if net is not None else \
        (lambda s: sbh.sbh_eval(t, Q, seed=s, opts=o, **gpu_kwargs(kind)))
    est = np.stack([f(s).cpu().numpy() for s in range(K)]).astype(np.float64)
    return est.var(0)


@pytest.mark.parametrize("kind", ["coulomb", "winding"])
def test_training_reduces_variance_on_held_out_queries(sbh, oracle_mod, kind):
    pts, w, nrm, q = _shapes(20000, 768, 47, kind)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    net = sbh.sbh_mlp_create(1)
    losses = sbh.sbh_mlp_train(net, t, dev(q[:512]), kernel=kind, steps=300, lr=3e-3)
    assert losses[-1] < 0.95 * losses[0], (losses[0], losses[-1])
    Q = dev(q[512:])
    for rr in (1, 0):  # roulette off (path sampling alone) and the paper's roulette
        v_mass = _variance(sbh, t, None, Q, kind, rr, 256)
        v_learn = _variance(sbh, t, net, Q, kind, rr, 256)
        print(kind, "rr", rr, "variance learned / mass", v_learn.sum() / v_mass.sum())
        assert v_learn.sum() < (0.7 if rr == 1 else 1.0) * v_mass.sum(), (rr, v_learn.sum(), v_mass.sum())
