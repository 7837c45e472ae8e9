"""Pins of the oracle's brute-force sum (Eq. 1) and kernels (Sec. 4.2, 4.3) by closed forms.

- Newton's shell theorem: a uniform spherical shell of mass M and radius R has potential M/|q|
  outside and M/R inside (Fibonacci-lattice quadrature, accurate to ~1e-6 at N = 4096).
- Gauss's law for the dipole kernel: oriented, area-weighted samples of a closed sphere have
  winding number 1 inside (at the centre every term equals a/(4 pi R^2)) and 0
  outside; the sign fixes the orientation (p - q) . n.
- One source: m / sqrt(r^2 + eps^2), and -log(m exp(-alpha r)) / alpha = r - log(m) / alpha.
- Log-sum-exp bound: with unit weights the smooth distance lies in [d_min - log(N)/alpha, d_min].
- Affine kernel: sum m (1 + g.(p - q)) = M + g.(sum m p - M q).
- Exact rounding: the compensated sum agrees with math.fsum of the same terms.
"""
import math

import numpy as np

from paper_2506_02219_gb300 import workloads as W

QS = np.array([[0, 0, 0], [0.3, 0.1, -0.2], [0.5, 0, 0], [2, 0, 0], [0, 3, 1], [-4, 2, 2]], np.float32)


def test_shell_theorem(oracle_mod):
    p, w, _ = W.sphere_fibonacci(4096, 1.0)
    w = (w / w.sum() * 3.0).astype(np.float32)
    M = float(w.astype(np.float64).sum())
    F = oracle_mod.brute(p, w, QS, oracle_mod.COULOMB, softening=0.0)
    r = np.linalg.norm(QS.astype(np.float64), axis=1)
    ref = np.where(r < 1.0, M / 1.0, M / np.maximum(r, 1e-30))
    np.testing.assert_allclose(F, ref, rtol=1e-5)


def test_gauss_winding_number(oracle_mod):
    p, w, nv = W.sphere_fibonacci(4096, 1.0)
    F = oracle_mod.brute(p, w, QS, oracle_mod.WINDING, normals=nv)
    inside = np.linalg.norm(QS, axis=1) < 1.0
    np.testing.assert_allclose(F[inside], 1.0, atol=1e-5)
    np.testing.assert_allclose(F[~inside], 0.0, atol=1e-5)
    # at the centre every term is a / (4 pi R^2) up to the FP32 rounding of p and n (~1e-7 each)
    assert abs(F[0] - float(w.astype(np.float64).sum()) / (4 * math.pi)) < 1e-7


def test_single_source_closed_forms(oracle_mod):
    p = np.array([[0.2, -0.1, 0.4]], np.float32)
    w = np.array([1.75], np.float32)
    q = np.array([[0.5, 0.3, -0.2], [0.2, -0.1, 0.4]], np.float32)
    r = np.linalg.norm(q.astype(np.float64) - p.astype(np.float64), axis=1)
    m = float(w[0])
    for eps in (0.0, 1e-3, 0.25):
        F = oracle_mod.brute(p, w, q[:1], oracle_mod.COULOMB, softening=eps)
        assert abs(F[0] - m / math.sqrt(r[0] ** 2 + eps * eps)) < 1e-15 * F[0]
    F = oracle_mod.brute(p, w, q, oracle_mod.SMOOTHDIST, alpha=7.0)
    d = -np.log(F) / 7.0
    np.testing.assert_allclose(d, r - math.log(m) / 7.0, rtol=0, atol=1e-14)


def test_smooth_distance_log_sum_exp_bound(oracle_mod):
    rng = np.random.default_rng(3)
    p = rng.random((500, 3)).astype(np.float32)
    w = np.ones(500, np.float32)
    q = rng.uniform(-0.5, 1.5, (50, 3)).astype(np.float32)
    for alpha in (20.0, 200.0):
        d = -np.log(oracle_mod.brute(p, w, q, oracle_mod.SMOOTHDIST, alpha=alpha)) / alpha
        dmin = np.min(np.linalg.norm(q[:, None, :].astype(np.float64) - p[None].astype(np.float64), axis=2), axis=1)
        assert np.all(d <= dmin + 1e-12)
        assert np.all(d >= dmin - math.log(500) / alpha - 1e-12)


def test_affine_kernel_closed_form(oracle_mod):
    rng = np.random.default_rng(4)
    p = rng.normal(size=(300, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 300).astype(np.float32)
    q = rng.normal(size=(20, 3)).astype(np.float32)
    g = (0.3, -0.7, 0.2)
    F = oracle_mod.brute(p, w, q, oracle_mod.AFFINE, affine=g)
    M = w.astype(np.float64).sum()
    mp = (w.astype(np.float64)[:, None] * p.astype(np.float64)).sum(0)
    ref = M + np.asarray(g) @ mp - M * (q.astype(np.float64) @ np.asarray(g))
    np.testing.assert_allclose(F, ref, rtol=1e-13)


def test_compensated_sum_is_exactly_rounded(oracle_mod):
    rng = np.random.default_rng(5)
    p = rng.random((2000, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, 2000).astype(np.float32)
    q = rng.random((5, 3)).astype(np.float32)
    F = oracle_mod.brute(p, w, q, oracle_mod.COULOMB, softening=1e-3)
    for j in range(5):
        d = p.astype(np.float64) - q[j].astype(np.float64)
        terms = w.astype(np.float64) / np.sqrt(np.sum(d * d, axis=1) + 1e-6)
        exact = math.fsum(terms.tolist())
        assert abs(F[j] - exact) <= 4e-16 * exact
