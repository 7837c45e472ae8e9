"""The learned child proposal on the GPU (a project extension of Sec. 3.3's path sampling).

- Scores of the tensor-core scorer (FP16 features, weights and hidden activations, FP32
  accumulation) against the oracle's FP64 network on the same FP16-rounded weights and features:
  the one rounding left, of the hidden activations to FP16 (relative 2^-11), moves a score by at
  most 2^-11 times the network's value on |weights| and |features|; the test allows 1e-3 of it.
- Training loss and gradient (FP32 master weights) against the oracle's FP64 loss and gradient,
  also with targets in the FP32 denormal range (the smooth distance's exp(-alpha r) residuals).
- Explicit training sets (features and |exact child residual| targets) against the oracle's
  features and brute-force residuals.
- Unbiasedness: seed-averaged learned estimates (both schedules, gate open everywhere and gated
  at one cell diagonal) within 4 sigma of the exact sum, sigma from the oracle's enumerated
  variance of the one-sample learned estimator with the same gate.
- near = 0 (gate closed) reproduces sbh_eval bit for bit.
- Training lowers the loss, and the trained proposal has lower variance than the mass-proportional
  pick on held-out queries.
"""
import numpy as np
import pytest

from gpu_util import dev, gpu_kwargs, oracle_kwargs, parity_error

pytestmark = pytest.mark.gpu


def _rand_weights(oracle_mod, seed, scale=0.3):
    return np.random.default_rng(seed).normal(scale=scale, size=oracle_mod.MLP_NPARAM).astype(np.float32)


def test_scores_match_oracle(sbh, oracle_mod):
    w = _rand_weights(oracle_mod, 1)
    net = sbh.sbh_mlp_create(0)
    sbh.sbh_mlp_set_weights(net, w)
    rng = np.random.default_rng(2)
    x = rng.normal(scale=3.0, size=(5003, 6)).astype(np.float32)  # a ragged last chunk of 32 rows
    g = sbh.sbh_mlp_scores(net, dev(x)).cpu().numpy().astype(np.float64)
    wh = w.astype(np.float16).astype(np.float64)
    xh = x.astype(np.float16).astype(np.float64)
    ref = oracle_mod.mlp_forward(wh, xh)
    scale = oracle_mod.mlp_forward(np.abs(wh), np.abs(xh))
    err = np.abs(g - ref) / scale
    assert np.all(err <= 1e-3), np.max(err)
    assert np.median(err) < 2e-4  # the bound is loose: typical errors are far inside it


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


def test_loss_grad_for_denormal_targets(sbh, oracle_mod):
    """The smooth distance's training targets exp(-alpha r) can be FP32 denormals, whose sum has no
    finite reciprocal. The loss depends only on each set's normalised targets, so targets scaled
    into the denormal range (1e-40) must give the loss and gradient of the unscaled ones, up to the
    denormals' rounding."""
    import torch
    sizes = [2, 5, 17, 64, 33]
    rng = np.random.default_rng(12)
    w = _rand_weights(oracle_mod, 5)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    x = rng.normal(size=(off[-1], 6)).astype(np.float32)
    t = rng.random(off[-1]).astype(np.float32)
    tiny = (t.astype(np.float64) * 1e-40).astype(np.float32)
    sums = [tiny[off[i]:off[i + 1]].astype(np.float64).sum() for i in range(len(sizes))]
    assert np.all(tiny < np.finfo(np.float32).tiny) and min(sums) < 1.0 / np.finfo(np.float32).max
    net = sbh.sbh_mlp_create(0)
    sbh.sbh_mlp_set_weights(net, w)
    loss, grad = sbh.sbh_mlp_loss_grad(net, dev(x), dev(tiny), torch.from_numpy(off).cuda())
    ref_loss, ref_g = oracle_mod.mlp_loss_grad(w.astype(np.float64), x.astype(np.float64), t.astype(np.float64), off)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.isfinite(float(loss.item())) and np.all(np.isfinite(g))
    assert abs(float(loss.item()) - ref_loss) <= 1e-3 * abs(ref_loss)
    assert np.max(np.abs(g - ref_g)) <= 1e-3 * np.max(np.abs(ref_g)), np.max(np.abs(g - ref_g)) / np.max(np.abs(ref_g))


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
@pytest.mark.parametrize("schedule,near", [(0, np.inf), (0, 1.0), (1, 1.0)])
def test_learned_seed_mean_within_four_sigma(sbh, oracle_mod, kind, schedule, near):
    pts, w, nrm, q = _shapes(400, 10, 41, kind)
    kw = oracle_kwargs(oracle_mod, kind, alpha=30.0)
    wt = _rand_weights(oracle_mod, 5, 0.5)
    ot = oracle_mod.Tree(pts, w, nrm, leaf_size=1, d=4)
    F = oracle_mod.brute(pts, w, q, normals=nrm, **kw)
    _, var = ot.enumerate_learned(q, wt.astype(np.float16).astype(np.float64), 0.1, near=near, **kw)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    net = sbh.sbh_mlp_create(0)
    sbh.sbh_mlp_set_weights(net, wt)
    o = sbh.eval_opts(raw_sum=1, schedule=schedule)
    Q = dev(q)
    K = 2000
    est = np.stack([sbh.sbh_eval_learned(t, net, Q, seed=s, opts=o, near=near, **gpu_kwargs(kind, alpha=30.0))
                    .cpu().numpy() for s in range(K)]).astype(np.float64)
    sigma = np.sqrt(np.maximum(var, 0.0) / K)
    dev_ = np.abs(est.mean(0) - F)
    assert np.all(dev_ <= 4 * sigma + 2e-6 * np.abs(F) + 1e-7), dev_ / np.maximum(sigma, 1e-30)
    if kind == "affine":  # zero variance under any proposal
        assert np.all(np.abs(est - F) <= 1e-4 * np.abs(F))


@pytest.mark.parametrize("kind", ["coulomb", "winding"])
@pytest.mark.parametrize("schedule", [0, 1])
def test_closed_gate_is_the_mass_estimator(sbh, oracle_mod, kind, schedule):
    pts, w, nrm, q = _shapes(6000, 777, 42, kind)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    net = sbh.sbh_mlp_create(3)
    o = sbh.eval_opts(schedule=schedule)
    a = sbh.sbh_eval_learned(t, net, dev(q), seed=9, opts=o, near=0.0, **gpu_kwargs(kind)).cpu().numpy()
    b = sbh.sbh_eval(t, dev(q), seed=9, opts=o, **gpu_kwargs(kind)).cpu().numpy()
    # same paths; the path probability is a product of FP32 mass fractions instead of m_T / m_a,
    # so the two differ by rounding, on the scale A of the terms (the oracle replay's abs_sum)
    _, A = oracle_mod.Tree(pts, w, nrm, leaf_size=1, d=4).replay(q, S=1, seed=9, return_abs_sum=True,
                                                                 **oracle_kwargs(oracle_mod, kind))
    err = parity_error(kind, a, b, A)
    assert np.mean(err <= 1e-5) >= 0.999, np.sort(err)[-5:]


def test_dataset_matches_oracle_residuals(sbh, oracle_mod):
    import torch
    kind = "winding"
    pts, w, nrm, q = _shapes(3000, 6, 43, kind)
    kw = oracle_kwargs(oracle_mod, kind)
    ot = oracle_mod.Tree(pts, w, nrm, leaf_size=1, d=4)
    e = ot.export()
    nodes = [v for v in np.nonzero((e["nchild"] >= 2) & (e["nchild"] <= 64))[0]][:40]
    set_q = np.repeat(np.arange(q.shape[0]), len(nodes)).astype(np.int32)
    set_node = np.tile(np.array(nodes), q.shape[0]).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(e["nchild"][set_node])]).astype(np.int64)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    feats, targ = sbh.sbh_mlp_dataset(t, dev(q), torch.from_numpy(set_q).cuda(), torch.from_numpy(set_node).cuda(),
                                      torch.from_numpy(off).cuda(), kernel=kind)
    feats, targ = feats.cpu().numpy(), targ.cpu().numpy()
    order = e["perm"]
    spts, sw, snrm = pts[order], w[order], nrm[order]
    for s_ in range(len(set_node)):
        j, a = int(set_q[s_]), int(set_node[s_])
        x = ot.child_features(a, q[j], True)
        np.testing.assert_allclose(feats[off[s_]:off[s_ + 1]], x, rtol=1e-4, atol=1e-4)
        f = int(e["first_child"][a])
        for c in range(int(e["nchild"][a])):
            b, en = int(e["begin"][f + c]), int(e["end"][f + c])
            exact = oracle_mod.brute(spts[b:en], sw[b:en], q[j:j + 1], normals=snrm[b:en], **kw)[0]
            # the child's own term at its FP32 centre of mass: its dipole sum(m n) for winding numbers
            own = oracle_mod.brute(e["com"][f + c:f + c + 1].astype(np.float32), np.ones(1, np.float32),
                                   q[j:j + 1], normals=e["dip"][f + c:f + c + 1].astype(np.float32), **kw)[0]
            scale = oracle_mod.brute(spts[b:en], sw[b:en], q[j:j + 1], normals=np.abs(snrm[b:en]), **kw)[0]
            assert abs(targ[off[s_] + c] - abs(exact - own)) <= 1e-5 * (abs(scale) + abs(own)) + 1e-12


def test_training_lowers_the_loss(sbh, oracle_mod):
    pts, w, nrm, q = _shapes(8000, 256, 44, "coulomb")
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    net = sbh.sbh_mlp_create(2)
    losses = sbh.sbh_mlp_train(net, t, dev(q), kernel="coulomb", near=2.0, steps=200, lr=3e-3)
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.95 * losses[0], (losses[0], losses[-1])
    _, step = sbh.sbh_mlp_get_weights(net)
    assert step == 200
    with pytest.raises(sbh.SBHError):  # no node within reach
        sbh.sbh_mlp_train(net, t, dev(q), kernel="coulomb", near=0.0, steps=1)


def _variance(sbh, t, net, Q, kind, rr, K, near=np.inf):
    o = sbh.eval_opts(rr=rr, raw_sum=1)
    f = (lambda s: sbh.sbh_eval_learned(t, net, Q, seed=s, opts=o, near=near, **gpu_kwargs(kind))) \
        if net is not None else (lambda s: sbh.sbh_eval(t, Q, seed=s, opts=o, **gpu_kwargs(kind)))
    est = np.stack([f(s).cpu().numpy() for s in range(K)]).astype(np.float64)
    return est.var(0)


@pytest.mark.parametrize("kind", ["coulomb", "winding"])
def test_training_reduces_variance_on_held_out_queries(sbh, oracle_mod, kind):
    pts, w, nrm, q = _shapes(20000, 768, 47, kind)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    Q = dev(q[512:])
    for near in (np.inf, 2.0):
        net = sbh.sbh_mlp_create(1)
        losses = sbh.sbh_mlp_train(net, t, dev(q[:512]), kernel=kind, near=near, steps=300, lr=3e-3)
        assert losses[-1] < 0.95 * losses[0], (losses[0], losses[-1])
        for rr in (1, 0):  # roulette off (path sampling alone) and the paper's roulette
            v_mass = _variance(sbh, t, None, Q, kind, rr, 256)
            v_learn = _variance(sbh, t, net, Q, kind, rr, 256, near)
            print(kind, "near", near, "rr", rr, "variance learned / mass", v_learn.sum() / v_mass.sum())
            assert v_learn.sum() < (0.7 if rr == 1 else 1.0) * v_mass.sum(), (near, rr, v_learn.sum(), v_mass.sum())


def test_checkpoint_resumes_training(sbh, oracle_mod, tmp_path):
    # 60 steps, checkpoint, 60 more on a restored copy == 120 steps straight, bit for bit (the
    # training sets come from a fixed stream and the gradient is summed in a fixed order)
    pts, w, nrm, q = _shapes(6000, 128, 45, "coulomb")
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm))
    Q = dev(q)
    a = sbh.sbh_mlp_create(4)
    sbh.sbh_mlp_train(a, t, Q, kernel="coulomb", near=2.0, steps=120, lr=3e-3)
    b = sbh.sbh_mlp_create(4)
    sbh.sbh_mlp_train(b, t, Q, kernel="coulomb", near=2.0, steps=60, lr=3e-3)
    path = str(tmp_path / "ckpt.npz")
    sbh.save_mlp(b, path)
    c = sbh.load_mlp(path)
    assert sbh.sbh_mlp_get_state(c)["adam_step"] == 60
    sbh.sbh_mlp_train(c, t, Q, kernel="coulomb", near=2.0, steps=60, lr=3e-3)
    wa, sa = sbh.sbh_mlp_get_weights(a)
    wc, sc = sbh.sbh_mlp_get_weights(c)
    assert sa == sc == 120
    assert np.array_equal(wc, wa)
