"""The seeded synthetic inputs: deterministic, in range, and the heavier-source option."""
import numpy as np

from paper_2506_02219_gb300 import workloads as W


def test_shape_union_is_deterministic_and_in_range():
    a = W.shape_union(3000, 11, n_ellipsoids=4, n_boxes=2)
    b = W.shape_union(3000, 11, n_ellipsoids=4, n_boxes=2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    p, w, n = a
    assert p.shape == (3000, 3) and w.shape == (3000,) and n.shape == (3000, 3)
    assert np.all(np.abs(p) <= 1.0) and np.all(w > 0)
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-5)


def test_single_ellipsoid_weights_sum_to_its_area():
    # one shape, nothing dropped: the area weights add up to the shape's area; for an ellipsoid
    # Thomsen's formula is within 1.1% of it
    p, w, n = W.shape_union(20000, 5, n_ellipsoids=1, rescale=False)
    # recover the semi-axes from the sample's extent along its principal axes
    c = p.mean(0)
    _, _, vt = np.linalg.svd(p - c, full_matrices=False)
    ext = np.abs((p - c) @ vt.T).max(0)
    a, b, cc = ext
    k = 1.6075
    thomsen = 4 * np.pi * (((a * b) ** k + (a * cc) ** k + (b * cc) ** k) / 3) ** (1 / k)
    assert abs(w.astype(np.float64).sum() / thomsen - 1) < 0.02


def test_heavier_sources_option():
    p0, w0, _ = W.shape_union(4000, 9, n_ellipsoids=3)
    p1, w1, _ = W.shape_union(4000, 9, n_ellipsoids=3, heavy_fraction=0.1)
    assert np.array_equal(p0, p1)
    ratio = w1 / w0
    heavy = np.isclose(ratio, 5.0, rtol=1e-6)
    assert heavy.sum() == 400 and np.allclose(ratio[~heavy], 1.0)


def test_far_field_queries_lie_outside_the_sources():
    wl = W.far_field_coulomb(n_sources=5000, res=40)
    assert wl.kernel == "coulomb" and wl.points.shape == (5000, 3)
    assert np.all(np.abs(wl.queries).max(1) > 1.2) and np.all(np.abs(wl.queries) <= 3.0)
    assert np.all(np.abs(wl.points) <= 1.0)


def test_random_order_winding_queries_share_the_grid_workloads_sources():
    a = W.winding_ellipsoids(n_sources=4096, grid=8)
    b = W.winding_ellipsoids_random(n_sources=4096, n_queries=5000)
    assert np.array_equal(a.points, b.points) and np.array_equal(a.weights, b.weights)
    lo, hi = a.points.min(0), a.points.max(0)
    assert b.queries.shape == (5000, 3) and np.all(b.queries >= lo) and np.all(b.queries <= hi)
    # unsorted: consecutive queries are as far apart as independent uniform draws
    step = np.linalg.norm(np.diff(b.queries, axis=0), axis=1).mean()
    assert step > 0.3 * np.linalg.norm(hi - lo)
