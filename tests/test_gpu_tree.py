"""GPU tree build (sbh_build) against the oracle's tree: identical structure (bit-exact integer
arrays: permutation, codes, node ranges, children, levels), FP64 aggregates within 1e-12, FP32
records equal to the FP64 values rounded, identical child-pick fractions, and the child pick's
guide table checked against its definition."""
import json
import os

import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_trees.json")


def compare_trees(g, o, d):
    np.testing.assert_array_equal(g["perm"], o["perm"])
    np.testing.assert_array_equal(g["code"], o["code"])
    N = o["begin"].shape[0]
    assert g["info"]["n_nodes"] == N
    for k in ("begin", "end", "first_child", "nchild", "level"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    # parent links are the inverse of the child ranges
    par = np.full(N, -1)
    for v in np.nonzero(o["nchild"])[0]:
        par[o["first_child"][v]:o["first_child"][v] + o["nchild"][v]] = v
    np.testing.assert_array_equal(g["parent"], par)
    np.testing.assert_allclose(g["com_mass64"][:, 3], o["mass"], rtol=1e-12)
    np.testing.assert_allclose(g["com_mass64"][:, :3], o["com"], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(g["com_mass"][:, 3], o["mass"].astype(np.float32))
    same = g["com_mass"][:, :3] == o["com"].astype(np.float32)
    assert same.mean() > 0.9999 and np.allclose(g["com_mass"][:, :3], o["com"], rtol=1e-6, atol=1e-7)
    assert (g["cdf"] == o["cdf"]).mean() > 0.9999 and np.allclose(g["cdf"], o["cdf"], rtol=1e-6)


def check_guide(g, rng):
    """The child pick's guide: entry of slot j of a node with nc children = the number of the
    first nc - 1 children's cdf values <= u_j, u_j = ceil(j 2^24 / nc) 2^-24; and a scan that starts
    there and steps up while cdf <= u gives the full count for any 24-bit u in slot j."""
    nch, fc, cdf, gd = g["nchild"], g["first_child"], g["cdf"], g["guide"]
    assert gd[0] == 0
    for v in np.nonzero(nch)[0]:
        f, nc = int(fc[v]), int(nch[v])
        c = cdf[f:f + nc - 1]
        j = np.arange(nc, dtype=np.int64)
        uj = ((j << 24) + nc - 1) // nc * np.float32(2.0 ** -24)
        want = (c[None, :] <= uj.astype(np.float32)[:, None]).sum(1)
        np.testing.assert_array_equal(gd[f:f + nc], want, err_msg=f"node {v}")
        m = rng.integers(0, 1 << 24, 64, dtype=np.int64)
        u = (m.astype(np.float32) * np.float32(2.0 ** -24))
        for mi, ui in zip(m, u):
            i = int(gd[f + ((mi * nc) >> 24)])
            while i < nc - 1 and c[i] <= ui:
                i += 1
            assert i == int((c <= ui).sum()), (v, mi)


def _build_both(sbh, oracle_mod, pts, w, nrm=None, leaf=1):
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm), leaf_size=leaf)
    # the 8-ary tree is built on the first Barnes-Hut call
    sbh.sbh_eval_bh(t, dev(pts[:1]), "coulomb", theta=0.5)
    return t, oracle_mod.Tree(pts, w, nrm, leaf_size=leaf, d=4), oracle_mod.Tree(pts, w, nrm, leaf_size=leaf, d=2)


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_hand_built_trees(sbh, case):
    pts = np.array(case["points"], np.float32)
    w = np.array(case["weights"], np.float32)
    t = sbh.sbh_build(dev(pts), dev(w), leaf_size=case["leaf_size"])
    if case["d"] == 2:
        sbh.sbh_eval_bh(t, dev(pts[:1]), "coulomb", theta=0.5)
    g = sbh.sbh_tree_export(t, 0 if case["d"] == 4 else 1)
    for k in ("perm", "begin", "end", "first_child", "nchild", "level"):
        np.testing.assert_array_equal(g[k], case[k], err_msg=k)
    np.testing.assert_allclose(g["com_mass"][:, 3], case["mass"], rtol=1e-7)
    np.testing.assert_array_equal(g["cdf"], np.array(case["cdf"], np.float32))
    assert g["info"]["n_sub"] == case["n_sub"] and g["info"]["first_sub"] == case["first_sub"]


@pytest.mark.parametrize("leaf", [1, 2, 7])
@pytest.mark.parametrize("kind,n", [("uniform", 4096), ("uniform", 5000), ("clustered", 20001), ("dups", 3000),
                                    ("shapes", 1 << 15)])
def test_tree_matches_oracle(sbh, oracle_mod, kind, n, leaf):
    rng = np.random.default_rng(n + leaf)
    nrm = None
    if kind == "uniform":
        pts = rng.random((n, 3)).astype(np.float32)
        w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    elif kind == "clustered":
        c = rng.normal(size=(7, 3))
        pts = (c[rng.integers(0, 7, n)] + 10 ** rng.uniform(-6, -1, (n, 1)) * rng.normal(size=(n, 3))).astype(np.float32)
        w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    elif kind == "dups":
        base = rng.random((900, 3)).astype(np.float32)
        pts = base[rng.integers(0, 900, n)]
        w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    else:
        from paper_2506_02219_gb300 import workloads as W
        pts, w, nrm = W.shape_union(n, 77, n_ellipsoids=8, n_boxes=2)
    t, o4, o2 = _build_both(sbh, oracle_mod, pts, w, nrm, leaf)
    g4 = sbh.sbh_tree_export(t, 0)
    compare_trees(g4, o4.export(), 4)
    compare_trees(sbh.sbh_tree_export(t, 1), o2.export(), 2)
    check_guide(g4, rng)
    if nrm is not None:
        g = sbh.sbh_tree_export(t, 0)
        np.testing.assert_allclose(g["dipole"], o4.export()["dip"], rtol=1e-5, atol=1e-9)


def test_tree_rebuild_is_bitwise_reproducible(sbh):
    rng = np.random.default_rng(1)
    pts = rng.random((30000, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 30000).astype(np.float32)
    a = sbh.sbh_tree_export(sbh.sbh_build(dev(pts), dev(w)), 0)
    b = sbh.sbh_tree_export(sbh.sbh_build(dev(pts), dev(w)), 0)
    for k in ("perm", "begin", "first_child", "com_mass", "cdf", "guide"):
        np.testing.assert_array_equal(a[k], b[k])
