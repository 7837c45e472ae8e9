"""sbh_solve_host: the one-shot build and evaluation from host buffers. Its output must equal
sbh_build + sbh_eval on device copies of the same data bit for bit (each chunk draws the random
stream of its place in the whole query set), for pinned and pageable host memory, chunk sizes that
leave a ragged last chunk, and every kernel; host-buffer misuse is rejected."""
import numpy as np
import pytest

from gpu_util import dev, gpu_kwargs

pytestmark = pytest.mark.gpu


def _data(kind, n=20000, nq=70001, seed=5):
    from paper_2506_02219_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    pts, w, nrm = W.shape_union(n, seed, n_ellipsoids=4, n_boxes=1)
    if kind != "winding":
        nrm = None
    if kind == "smoothdist":
        w = np.ones_like(w)
    q = rng.uniform(-1.05, 1.05, (nq, 3)).astype(np.float32)
    return pts, w, nrm, q


@pytest.mark.parametrize("kind", ["coulomb", "winding", "smoothdist", "affine"])
@pytest.mark.parametrize("chunk", [0, 9999, 70001])
def test_host_solve_equals_device_path(sbh, kind, chunk):
    pts, w, nrm, q = _data(kind)
    t = sbh.sbh_build(dev(pts), dev(w), dev(nrm), leaf_size=2)
    ref = sbh.sbh_eval(t, dev(q), samples_per_subdomain=2, seed=77, **gpu_kwargs(kind)).cpu().numpy()
    out = sbh.sbh_solve_host(pts, w, q, normals=nrm, leaf_size=2, samples_per_subdomain=2, seed=77, chunk=chunk,
                             **gpu_kwargs(kind))
    assert np.array_equal(out, ref, equal_nan=True)


def test_host_solve_with_pinned_buffers_and_options(sbh):
    import torch
    pts, w, nrm, q = _data("coulomb", nq=3 * (1 << 20) + 17)
    o = sbh.eval_opts(rr=2, schedule=1)
    t = sbh.sbh_build(dev(pts), dev(w))
    ref = sbh.sbh_eval(t, dev(q), seed=9, opts=o).cpu().numpy()
    P, M, Q = (torch.from_numpy(x).pin_memory() for x in (pts, w, q))
    out = torch.empty(q.shape[0], dtype=torch.float32).pin_memory()
    sbh.sbh_solve_host(P, M, Q, seed=9, opts=o, out=out)
    assert np.array_equal(out.numpy(), ref)


def test_host_solve_rejects_device_buffers(sbh):
    pts, w, nrm, q = _data("coulomb", n=500, nq=10)
    with pytest.raises(ValueError):
        sbh.sbh_solve_host(dev(pts), w, q)
    with pytest.raises(sbh.SBHError):
        sbh.sbh_solve_host(pts, w, q, kernel="winding")  # no normals
