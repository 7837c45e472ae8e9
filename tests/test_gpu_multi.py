"""Many independent problems in one persistent launch (sbh_multi_plan_*), its CUDA-graph capture,
the one-thread-per-query schedule, and the autotuner."""
import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu

SIZES = [(1, 0), (7, 1), (300, 31), (5000, 33), (70000, 1000), (1 << 17, 50000), (3, 5), (2049, 0), (40000, 777)]


def _sets(kind="coulomb", sizes=SIZES, seed=5):
    from paper_2506_02219_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    out = []
    for i, (n, nq) in enumerate(sizes):
        if kind == "winding" and n >= 64:
            p, w, nv = W.shape_union(n, seed + i, n_ellipsoids=3, n_boxes=1)
        else:
            p = rng.normal(size=(n, 3)).astype(np.float32)
            w = rng.uniform(0.5, 1.5, n).astype(np.float32)
            nv = rng.normal(size=(n, 3)).astype(np.float32)
            nv /= np.linalg.norm(nv, axis=1, keepdims=True)
        q = rng.uniform(-1.5, 1.5, (nq, 3)).astype(np.float32)
        out.append((p, w, nv if kind == "winding" else None, q))
    return out


@pytest.mark.parametrize("kind,S", [("coulomb", 1), ("winding", 2), ("smoothdist", 1)])
def test_multi_launch_equals_per_set_evaluation(sbh, kind, S):
    import torch
    sets = _sets(kind)
    trees = [sbh.sbh_build(dev(p), dev(w), dev(nv)) for p, w, nv, _ in sets]
    Qs = [dev(q) if q.shape[0] else torch.zeros((0, 3), device="cuda") for *_, q in sets]
    plan = sbh.sbh_multi_plan_create(trees, Qs, kind, S, seed=11)
    outs = sbh.sbh_multi_plan_launch(plan)
    for t, Q, o in zip(trees, Qs, outs):
        if Q.shape[0] == 0:
            continue
        ref = sbh.sbh_eval(t, Q, kind, S, 11)
        torch.testing.assert_close(o, ref, rtol=0, atol=0, equal_nan=True)


def test_multi_launch_replays_from_a_cuda_graph(sbh):
    import torch
    sets = _sets("coulomb", seed=7)
    trees = [sbh.sbh_build(dev(p), dev(w)) for p, w, _, _ in sets]
    Qs = [dev(q) if q.shape[0] else torch.zeros((0, 3), device="cuda") for *_, q in sets]
    plan = sbh.sbh_multi_plan_create(trees, Qs, "coulomb", 1, seed=3)
    direct = [o.clone() for o in sbh.sbh_multi_plan_launch(plan)]
    graph = sbh.capture_multi(plan)
    assert graph.sbh_kernels == 1  # one persistent launch per replay
    for _ in range(3):
        for o in plan.outs:
            o.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip(direct, plan.outs):
            torch.testing.assert_close(a, b, rtol=0, atol=0)


def test_multi_plan_rejects_inconsistent_sets(sbh):
    p, w, _, q = _sets("coulomb", sizes=[(500, 10)])[0]
    t = sbh.sbh_build(dev(p), dev(w))
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_multi_plan_create([t], [dev(q)], "winding", 1)  # no normals
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_multi_plan_create([t], [dev(q)], "coulomb", 0)


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist"])
def test_thread_per_query_schedule_matches_replay(sbh, oracle_mod, kind):
    from gpu_util import gpu_kwargs, oracle_kwargs, parity_error
    sets = _sets("winding" if kind == "winding" else "coulomb", sizes=[(20000, 3001)], seed=13)
    p, w, nv, q = sets[0]
    t = sbh.sbh_build(dev(p), dev(w), dev(nv))
    o = sbh.eval_opts(schedule=1)
    g = sbh.sbh_eval(t, dev(q), seed=21, opts=o, **gpu_kwargs(kind)).cpu().numpy()
    r, A = oracle_mod.Tree(p, w, nv).replay(q, seed=21, return_abs_sum=True, **oracle_kwargs(oracle_mod, kind))
    err = parity_error(kind, g, r, A)
    assert np.mean(err <= 1e-4) >= 0.999


def test_autotuner_picks_a_measured_configuration(sbh):
    from paper_2506_02219_gb300 import autotune
    from paper_2506_02219_gb300 import workloads as W
    p, w, nv = W.shape_union(1 << 16, 3, n_ellipsoids=6, n_boxes=2)
    q = np.random.default_rng(0).uniform(-1, 1, (1 << 16, 3)).astype(np.float32)
    r = autotune.autotune(dev(p), dev(w), dev(q), "coulomb", leaf_sizes=(1, 4), samples=(1, 2), schedules=(0, 1),
                          n_err_queries=2048)
    assert len(r["table"]) == 8
    assert r["best"] in r["table"]
    target = sorted(x["median_rel_err"] for x in r["table"])[4]
    r2 = autotune.autotune(dev(p), dev(w), dev(q), "coulomb", target_median_rel_err=target, leaf_sizes=(1, 4),
                           samples=(1, 2), schedules=(0, 1), n_err_queries=2048)
    assert r2["best"]["median_rel_err"] <= target
