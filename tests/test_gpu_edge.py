"""Edge cases and error behaviour of the C ABI on the GPU."""
import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu


def test_single_and_two_point_trees(sbh, oracle_mod):
    q = np.random.default_rng(0).random((37, 3)).astype(np.float32)
    for pts, w, leaf in [(np.array([[0.3, 0.2, 0.1]], np.float32), np.array([2.0], np.float32), 1),
                         (np.array([[0, 0, 0], [1, 0, 0]], np.float32), np.array([1.0, 3.0], np.float32), 2),
                         (np.array([[0, 0, 0], [1, 0, 0]], np.float32), np.array([1.0, 3.0], np.float32), 1)]:
        t = sbh.sbh_build(dev(pts), dev(w), leaf_size=leaf)
        F = oracle_mod.brute(pts, w, q)
        g = sbh.sbh_eval(t, dev(q), "coulomb", seed=3).cpu().numpy()
        np.testing.assert_allclose(g, F, rtol=1e-5)  # every subdomain is a point: exact
        b = sbh.sbh_eval_bh(t, dev(q), "coulomb", theta=0.0).cpu().numpy()
        np.testing.assert_allclose(b, F, rtol=1e-5)


def test_all_points_identical(sbh, oracle_mod):
    pts = np.tile(np.array([[0.5, 0.25, -1.0]], np.float32), (1000, 1))
    w = np.random.default_rng(2).uniform(0.5, 1.5, 1000).astype(np.float32)
    q = np.random.default_rng(3).random((100, 3)).astype(np.float32)
    t = sbh.sbh_build(dev(pts), dev(w))
    info = sbh.sbh_tree_info(t)
    assert info["n_sub"] == 1000 and info["side"] == 1.0
    F = oracle_mod.brute(pts, w, q)
    np.testing.assert_allclose(sbh.sbh_eval(t, dev(q), "coulomb").cpu().numpy(), F, rtol=1e-5)


def test_empty_and_ragged_query_sets(sbh, oracle_mod):
    rng = np.random.default_rng(4)
    pts = rng.random((5000, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 5000).astype(np.float32)
    t = sbh.sbh_build(dev(pts), dev(w))
    import torch
    out = sbh.sbh_eval(t, torch.zeros((0, 3), device="cuda"), "coulomb")
    assert out.shape == (0,)
    ot = oracle_mod.Tree(pts, w)
    for nq in (1, 31, 33, 257, 1025):
        q = rng.random((nq, 3)).astype(np.float32)
        g = sbh.sbh_eval(t, dev(q), "coulomb", seed=8).cpu().numpy()
        r = ot.replay(q, seed=8)
        assert np.all(np.abs(g - r) / r < 1e-4)


def test_invalid_arguments_are_rejected(sbh):
    rng = np.random.default_rng(5)
    pts = rng.random((100, 3)).astype(np.float32)
    w = np.ones(100, np.float32)
    bad = pts.copy()
    bad[7, 1] = np.nan
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_build(dev(bad), dev(w))
    bad = pts.copy()
    bad[3, 0] = np.inf
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_build(dev(bad), dev(w))
    for wv in (0.0, -1.0, np.nan):
        ww = w.copy()
        ww[11] = wv
        with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
            sbh.sbh_build(dev(pts), dev(ww))
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_build(dev(pts), dev(w), leaf_size=0)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_build(dev(pts), dev(w), leaf_size=65)
    t = sbh.sbh_build(dev(pts), dev(w))
    q = dev(pts[:10])
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval(t, q, "winding")  # no normals
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval(t, q, "coulomb", samples_per_subdomain=0)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval(t, q, "smoothdist", alpha=0.0)
    o = sbh.EvalOpts()
    o.rr = 7
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval(t, q, "coulomb", opts=o)
    with pytest.raises(sbh.SBHError, match="SBH_EINVAL"):
        sbh.sbh_eval_bh(t, q, "coulomb", theta=-1.0)


def test_host_pointers_are_rejected(sbh):
    import ctypes
    lib = sbh.load_library()
    host = np.zeros((10, 3), np.float32)
    hw = np.ones(10, np.float32)
    h = ctypes.c_void_p()
    st = lib.sbh_build(host.ctypes.data_as(ctypes.c_void_p), hw.ctypes.data_as(ctypes.c_void_p), None, 10, 1, None,
                       ctypes.byref(h))
    assert st == 1 and b"device memory" in lib.sbh_last_error()


def test_evaluation_is_bitwise_reproducible(sbh):
    rng = np.random.default_rng(6)
    pts = rng.random((20000, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 20000).astype(np.float32)
    q = dev(rng.random((5000, 3)).astype(np.float32))
    t = sbh.sbh_build(dev(pts), dev(w))
    a = sbh.sbh_eval(t, q, "coulomb", seed=5).cpu().numpy()
    b = sbh.sbh_eval(t, q, "coulomb", seed=5).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    assert np.any(a != sbh.sbh_eval(t, q, "coulomb", seed=6).cpu().numpy())
