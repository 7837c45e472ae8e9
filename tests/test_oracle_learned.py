"""Pins of the oracle's learned child proposal (a project extension of Sec. 3.3's path sampling).

- The network's loss gradient against central finite differences (FP64).
- A hand-built network with a closed-form score.
- Unbiasedness with any proposal that keeps every child probability > 0: the enumerated mean of the
  estimator with the learned proposal equals the brute-force sum to 1e-12, for random weights.
- The features are invariant to translating and scaling the whole problem.
"""
import numpy as np
import pytest

from test_oracle_estimator import KINDS, _setup


def test_loss_gradient_matches_finite_differences(oracle_mod):
    rng = np.random.default_rng(0)
    w = rng.normal(scale=0.3, size=oracle_mod.MLP_NPARAM)
    sizes = [2, 5, 17, 64]
    off = np.concatenate([[0], np.cumsum(sizes)])
    x = rng.normal(size=(off[-1], 6))
    t = rng.random(off[-1])
    loss, g = oracle_mod.mlp_loss_grad(w, x, t, off)
    idx = rng.choice(oracle_mod.MLP_NPARAM, 60, replace=False)
    idx = np.unique(np.concatenate([idx, [0, 191, 192, 223, 224, 1247, 1248, 1279, 1280, 1311, 1312]]))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(w)
        e[i] = h
        fd = (oracle_mod.mlp_loss_grad(w + e, x, t, off)[0] - oracle_mod.mlp_loss_grad(w - e, x, t, off)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()), (i, fd, g[i])


def test_hand_built_network(oracle_mod):
    w = np.zeros(oracle_mod.MLP_NPARAM)
    # W1 row 0 = e_0 (score path through hidden unit 0 of both layers), W2[0][0] = 1, w3[0] = 2, b3 = 0.5
    w[0] = 1.0
    w[192 + 32 + 0] = 1.0
    w[192 + 32 + 1024 + 32 + 0] = 2.0
    w[-1] = 0.5
    x = np.array([[0.7, 1, 2, 3, 4, 5], [-0.4, 1, 1, 1, 1, 1]])
    np.testing.assert_allclose(oracle_mod.mlp_forward(w, x), [2 * 0.7 + 0.5, 0.5], rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [9, 300])
@pytest.mark.parametrize("near", [np.inf, 1.0])
def test_learned_proposal_keeps_the_estimator_unbiased(oracle_mod, kind, n, near):
    t, q, F, kw = _setup(oracle_mod, n, 500 + n, kind)
    w = np.random.default_rng(n).normal(scale=0.5, size=oracle_mod.MLP_NPARAM)
    mean, var = t.enumerate_learned(q, w, 0.1, near=near, **kw)
    scale = np.maximum(np.abs(F), 1e-3 if kind == "winding" else 0.0)
    assert np.all(np.abs(mean - F) <= 1e-12 * scale + 1e-15)
    assert np.all(var >= -1e-12 * scale * scale)


def test_features_are_translation_and_scale_invariant(oracle_mod):
    rng = np.random.default_rng(1)
    pts = rng.random((500, 3))
    w = rng.uniform(0.5, 1.5, 500)
    nv = rng.normal(size=(500, 3))
    q = np.array([0.3, 0.7, 0.2])
    t1 = oracle_mod.Tree(pts.astype(np.float32), w.astype(np.float32), nv.astype(np.float32))
    # a power-of-two scale and a translation that keep the float32 points and codes exact
    t2 = oracle_mod.Tree((pts * 4 + 8).astype(np.float32), w.astype(np.float32), nv.astype(np.float32))
    e = t1.export()
    for node in np.nonzero(e["nchild"])[0][:20]:
        np.testing.assert_allclose(t1.child_features(node, q, True), t2.child_features(node, q * 4 + 8, True),
                                   rtol=1e-5, atol=1e-5)


def test_all_zero_targets_mean_no_preference(oracle_mod):
    # a decision set whose children all have zero residual gets uniform targets: with a network
    # that scores every child alike, the cross-entropy is log(nc) and the gradient vanishes
    w = np.zeros(oracle_mod.MLP_NPARAM)
    w[-1] = 0.3
    x = np.random.default_rng(2).normal(size=(7, 6))
    loss, g = oracle_mod.mlp_loss_grad(w, x, np.zeros(7), [0, 7])
    assert abs(loss - np.log(7)) <= 1e-15
    assert np.all(np.abs(g) <= 1e-15)


@pytest.mark.parametrize("kind", ["coulomb", "winding"])
def test_gate_closed_everywhere_is_the_mass_proposal(oracle_mod, kind):
    # near = 0: no node is near enough, every pick is mass-proportional and p(I in T) is the
    # product of the mass fractions, m_T / m_a: the variance is that of Algorithm 2 with mass p_agg
    t, q, F, kw = _setup(oracle_mod, 300, 77, kind)
    w = np.random.default_rng(3).normal(scale=0.5, size=oracle_mod.MLP_NPARAM)
    mean_l, var_l = t.enumerate_learned(q, w, 0.1, near=0.0, **kw)
    mean_m, var_m = t.enumerate(q, **kw)
    np.testing.assert_allclose(mean_l, mean_m, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(var_l, var_m, rtol=1e-9, atol=1e-12 * np.max(np.abs(F)) ** 2)


def test_gate_changes_the_variance_only_near_the_query(oracle_mod):
    # a query far from every subdomain (more than 1 diagonal away) sees the mass proposal for near = 1
    t, q, F, kw = _setup(oracle_mod, 300, 78, "coulomb")
    far = np.array([[9.0, 9.0, 9.0]], np.float32)
    w = np.random.default_rng(4).normal(scale=0.5, size=oracle_mod.MLP_NPARAM)
    _, v1 = t.enumerate_learned(far, w, 0.1, near=1.0, **kw)
    _, vm = t.enumerate(far, **kw)
    _, vi = t.enumerate_learned(far, w, 0.1, **kw)
    np.testing.assert_allclose(v1, vm, rtol=1e-9)
    assert abs(vi[0] - vm[0]) > 1e-6 * vm[0]
