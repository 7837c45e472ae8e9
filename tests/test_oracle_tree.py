"""Pins of the oracle's tree (Sec. 3.1): hand-derived cases (tests/golden/hand_trees.json) and the
invariants that define the structure on random inputs."""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_trees.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_built_trees(oracle_mod, case):
    t = oracle_mod.Tree(np.array(case["points"], np.float32), np.array(case["weights"], np.float32),
                        leaf_size=case["leaf_size"], d=case["d"])
    e = t.export()
    for key in ("perm", "begin", "end", "first_child", "nchild", "level"):
        np.testing.assert_array_equal(e[key], case[key], err_msg=key)
    np.testing.assert_allclose(e["mass"], case["mass"], rtol=1e-7)
    np.testing.assert_array_equal(e["cdf"], np.array(case["cdf"], np.float32))
    m = t.meta()
    assert m["n_sub"] == case["n_sub"] and m["first_sub"] == case["first_sub"]


def check_tree_invariants(e, pts, w, leaf_size, d):
    """Structure of the tree of Sec. 3.1 under the collapse and leaf readings."""
    n = pts.shape[0]
    bits = 6 if d == 4 else 3
    maxl = 60 // bits
    perm, code = e["perm"], e["code"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.all(code[1:] >= code[:-1])
    same = code[1:] == code[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])  # stable
    N = e["begin"].shape[0]
    b, en, fc, nc, lv = e["begin"], e["end"], e["first_child"], e["nchild"], e["level"]
    assert b[0] == 0 and en[0] == n
    next_fc = 1
    for v in range(N):
        cnt = en[v] - b[v]
        assert cnt >= 1
        if nc[v] == 0:
            assert cnt == 1
            continue
        assert nc[v] >= 2
        assert fc[v] == next_fc  # breadth-first, children contiguous
        next_fc += nc[v]
        kids = np.arange(fc[v], fc[v] + nc[v])
        assert b[kids[0]] == b[v] and en[kids[-1]] == en[v]
        assert np.all(b[kids[1:]] == en[kids[:-1]])
        assert np.all(lv[kids] > lv[v])
        is_leaf = cnt <= leaf_size or lv[v] == maxl
        if is_leaf:  # points as children, one level down
            assert np.all(en[kids] - b[kids] == 1) and np.all(lv[kids] == lv[v] + 1) and nc[v] == cnt
        else:
            assert cnt > leaf_size
            c = code[b[v]:en[v]]
            shift = np.uint64(60 - bits * lv[v])
            top = c >> shift if lv[v] > 0 else np.zeros_like(c)
            assert np.all(top == top[0])  # one cell at its level
            dig = (code[b[kids]] >> np.uint64(60 - bits * (lv[v] + 1))) & np.uint64((1 << bits) - 1)
            assert np.all(np.diff(dig.astype(np.int64)) > 0)  # distinct cells one level down, Morton order
            for k in kids:  # each child holds exactly one cell one level down
                ck = code[b[k]:en[k]] >> np.uint64(60 - bits * (lv[v] + 1))
                assert np.all(ck == ck[0])
    assert next_fc == N
    # aggregates
    m64 = w.astype(np.float64)[perm]
    p64 = pts.astype(np.float64)[perm]
    cs = np.concatenate([[0.0], np.cumsum(m64)])
    np.testing.assert_allclose(e["mass"], cs[en] - cs[b], rtol=1e-9)
    for v in range(0, N, max(1, N // 200)):
        mp = (m64[b[v]:en[v], None] * p64[b[v]:en[v]]).sum(0)
        np.testing.assert_allclose(e["com"][v] * e["mass"][v], mp, rtol=1e-9, atol=1e-12)
    for v in range(N):
        if nc[v]:
            kids = np.arange(fc[v], fc[v] + nc[v])
            pre = np.cumsum(e["mass"][kids]) / e["mass"][kids].sum()
            ref = pre.astype(np.float32)
            ref[-1] = 1.0
            np.testing.assert_array_equal(e["cdf"][kids], ref)


@pytest.mark.parametrize("d", [4, 2])
@pytest.mark.parametrize("leaf_size", [1, 3])
@pytest.mark.parametrize("kind", ["uniform", "clustered", "dups"])
def test_tree_invariants(oracle_mod, d, leaf_size, kind):
    rng = np.random.default_rng(11)
    if kind == "uniform":
        pts = rng.random((3000, 3)).astype(np.float32)
    elif kind == "clustered":
        c = rng.random((5, 3))
        pts = (c[rng.integers(0, 5, 3000)] + 1e-3 * rng.normal(size=(3000, 3))).astype(np.float32)
    else:
        base = rng.random((700, 3)).astype(np.float32)
        pts = base[rng.integers(0, 700, 2000)]
    w = rng.uniform(0.5, 1.5, pts.shape[0]).astype(np.float32)
    t = oracle_mod.Tree(pts, w, leaf_size=leaf_size, d=d)
    check_tree_invariants(t.export(), pts, w, leaf_size, d)
