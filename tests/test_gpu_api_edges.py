"""Edge cases of the entry points added beside sbh_build / sbh_eval: empty and one-point inputs,
rejected arguments, and the conventions of the brute-force gradient and the host-buffer call."""
import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu


def _cloud(n, nq, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.random((n, 3)).astype(np.float32), rng.uniform(0.5, 1.5, n).astype(np.float32),
            rng.random((nq, 3)).astype(np.float32))


def test_solve_host_empty_and_single_point(sbh):
    p, w, q = _cloud(1, 5)
    out = sbh.sbh_solve_host(p, w, q[:0])
    assert out.shape == (0,)
    out = sbh.sbh_solve_host(p, w, q)  # one source: the control variate is the exact sum
    ref = w[0] / np.sqrt(((p[0] - q) ** 2).sum(1) + 1e-6)
    np.testing.assert_allclose(out, ref, rtol=1e-5)


def test_solve_host_rejects_bad_arguments(sbh):
    p, w, q = _cloud(100, 10)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_solve_host(p, w, q, leaf_size=0)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_solve_host(p, -w, q)  # p_agg needs positive masses
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_solve_host(p, w, q, samples_per_subdomain=0)


def test_sample_count_beyond_the_tag_width_is_rejected(sbh):
    # the warp-task schedule carries the sample index in 16 bits: S = 2^16 is the largest accepted,
    # beyond it every entry point returns SBH_EINVAL before any launch
    p, w, q = _cloud(200, 8)
    t = sbh.sbh_build(dev(p), dev(w))
    Q = dev(q)
    big = (1 << 16) + 1
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval(t, Q, samples_per_subdomain=big)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval_grad(t, Q, samples_per_subdomain=big)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval_count(t, Q, samples_per_subdomain=big)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_solve_host(p, w, q, samples_per_subdomain=big)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_multi_plan_create([t], [Q], "coulomb", big)
    assert sbh.sbh_eval(t, Q[:1], samples_per_subdomain=1).shape == (1,)


def test_brute_grad_empty_sources_and_queries(sbh):
    import torch
    p, w, q = _cloud(0, 4)
    out, g = sbh.sbh_eval_brute_grad(dev(p).reshape(0, 3), dev(w), dev(q))
    assert torch.all(out == 0) and torch.all(g == 0)
    p, w, q = _cloud(10, 0)
    out, g = sbh.sbh_eval_brute_grad(dev(p), dev(w), dev(q).reshape(0, 3))
    assert out.numel() == 0 and g.numel() == 0


def test_brute_grad_single_source_closed_form(sbh):
    p = np.array([[0.3, -0.2, 0.5]], np.float32)
    w = np.array([2.0], np.float32)
    q = np.array([[1.0, 1.0, 1.0], [-0.5, 0.2, 0.1]], np.float32)
    _, g = sbh.sbh_eval_brute_grad(dev(p), dev(w), dev(q), softening=0.0)
    d = (p[0] - q).astype(np.float64)
    ref = 2.0 * d / (np.linalg.norm(d, axis=1) ** 3)[:, None]  # grad_q m / |p - q|
    np.testing.assert_allclose(g.cpu().numpy(), ref, rtol=1e-5)


def test_learned_entry_points_reject_bad_arguments(sbh):
    p, w, q = _cloud(2000, 10)
    t = sbh.sbh_build(dev(p), dev(w))
    net = sbh.sbh_mlp_create(0)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval_learned(t, net, dev(q), opts=sbh.eval_opts(sampling=1))
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval_learned(t, net, dev(q), near=-1.0)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_mlp_train(net, t, dev(q), near=-1.0, steps=1)
    with pytest.raises(ValueError):
        sbh.sbh_mlp_set_weights(net, np.zeros(10, np.float32))
    st = sbh.sbh_mlp_get_state(net)
    assert st["adam_step"] == 0 and st["weights"].shape == (sbh.MLP_PARAMS,)
    with pytest.raises(ValueError):
        sbh.sbh_mlp_set_state(net, {"weights": st["weights"][:5], "adam_m": st["adam_m"], "adam_v": st["adam_v"],
                                    "adam_step": 0})


def test_memory_returns_to_baseline_after_every_entry_point(sbh):
    import torch
    p, w, q = _cloud(5000, 3000)
    torch.cuda.synchronize()
    base = sbh.sbh_memory_in_use()
    t = sbh.sbh_build(dev(p), dev(w))
    sbh.sbh_eval(t, dev(q))
    sbh.sbh_eval_grad(t, dev(q))
    sbh.sbh_eval_bh(t, dev(q))
    net = sbh.sbh_mlp_create(0)
    sbh.sbh_mlp_train(net, t, dev(q[:64]), near=2.0, steps=2)
    sbh.sbh_eval_learned(t, net, dev(q), near=1.0)
    plan = sbh.sbh_multi_plan_create([t], [dev(q)], "coulomb", 1)
    sbh.sbh_multi_plan_launch(plan)
    sbh.sbh_multi_plan_free(plan)
    net.free()
    t.free()
    sbh.sbh_solve_host(p, w, q)
    torch.cuda.synchronize()
    assert sbh.sbh_memory_in_use() == base
