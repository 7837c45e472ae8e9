"""Pins of the oracle's query gradients (the adjoint of the estimator under a fixed random stream).

- Brute-force gradient of Eq. 1 against central finite differences of the brute-force sum.
- The estimator applied to grad_q f with the same paths and weights is unbiased: its enumerated
  mean equals the brute-force gradient to 1e-12 (the theorem of Appendix A for a vector kernel).
- The adjoint is the derivative of the frozen-path estimate: central differences of the estimate
  along the paths drawn at q (values at q +- h) match the replayed gradient.
- Along its own paths, the gradient replay's value equals the plain replay.
"""
import numpy as np
import pytest

from test_oracle_estimator import KINDS, _setup

H = 1e-5


def _fd(fn, q, h):
    g = np.zeros((q.shape[0], 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        g[:, a] = (fn(q + e) - fn(q - e)) / (2 * h)
    return g


@pytest.mark.parametrize("kind", KINDS)
def test_brute_gradient_matches_finite_differences(oracle_mod, kind):
    t, q, F, kw = _setup(oracle_mod, 200, 41, kind)
    q = q[:6].astype(np.float64)
    G = oracle_mod.brute_grad(t.points, t.weights, q, normals=t.normals, **kw)
    # the finite differences need FP64 query positions, which the oracle's brute force (float32
    # queries, like the GPU) does not take: the sums of Eq. 1 are evaluated here in numpy; their
    # value formulas are pinned by the closed-form tests of test_oracle_brute.py
    pts, w, nrm = t.points, t.weights, t.normals

    def F64(qq):
        out = np.zeros(qq.shape[0])
        for j, x in enumerate(qq):
            d = pts.astype(np.float64) - x
            r2 = (d * d).sum(1)
            r = np.sqrt(r2)
            m = w.astype(np.float64)
            if kind == "coulomb":
                out[j] = (m / np.sqrt(r2 + 1e-6)).sum()
            elif kind == "winding":
                N = m[:, None] * nrm.astype(np.float64)
                out[j] = ((d * N).sum(1) / (4 * np.pi * r2 * r)).sum()
            elif kind == "smoothdist":
                out[j] = (m * np.exp(-30.0 * r)).sum()
            else:
                out[j] = (m * (1 + d @ np.array([0.4, -0.3, 0.8]))).sum()
        return out

    fd = _fd(F64, q, H)
    scale = np.abs(G).max(1, keepdims=True) + 1e-12
    assert np.all(np.abs(fd - G) <= 1e-5 * scale), np.abs(fd - G).max()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("sampling,rr", [(0, 0), (1, 0), (0, 1), (0, 2)])
def test_gradient_estimator_is_unbiased(oracle_mod, kind, sampling, rr):
    t, q, F, kw = _setup(oracle_mod, 300, 42, kind)
    G = oracle_mod.brute_grad(t.points, t.weights, q, normals=t.normals, **kw)
    E = t.enumerate_grad(q, sampling=sampling, rr=rr, **kw)
    scale = np.abs(G).max(1, keepdims=True) + 1e-3 * (kind == "winding")
    assert np.all(np.abs(E - G) <= 1e-11 * scale + 1e-14)


@pytest.mark.parametrize("kind", KINDS)
def test_adjoint_is_the_frozen_path_derivative(oracle_mod, kind):
    t, q, F, kw = _setup(oracle_mod, 300, 43, kind)
    q = q[:6]
    for seed in (3, 9):
        val, G, A = t.replay_grad(q, S=2, seed=seed, **kw)
        np.testing.assert_allclose(val, t.replay(q, S=2, seed=seed, **kw), rtol=1e-12, atol=1e-14)

        def frozen(qq, seed=seed):
            return t.replay_grad(q, S=2, seed=seed, eval_at=qq, **kw)[0]

        fd = _fd(frozen, q.astype(np.float64), 1e-6)
        assert np.all(np.abs(fd - G) <= 1e-5 * A[:, None] + 1e-12), np.abs(fd - G).max()
