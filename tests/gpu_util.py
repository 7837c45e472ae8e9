"""Helpers shared by the GPU parity tests."""
import numpy as np

KIND_ID = {"coulomb": 0, "winding": 1, "smoothdist": 2, "affine": 3}
AFFINE_G = (0.4, -0.3, 0.8)


def dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def parity_error(kind, gpu, ref, abs_sum, alpha=200.0):
    """Per-query error of a GPU estimate against the oracle's replay of the same random stream:
    |F_gpu - F_oracle| / A, with A the sum of the absolute values of every term the estimate adds
    (the oracle's abs_sum; A >= |F|, and A is the scale of the rounding error of any evaluation of
    the same signed sum), at least 1 for winding numbers. For the smooth distance the GPU returns
    d = -log(F_gpu) / alpha, +inf where its estimate of F is <= 0; that matches an oracle estimate
    <= 0."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.asarray(abs_sum, np.float64)
    inf_out = np.isposinf(gpu)
    if kind == "smoothdist":
        gpu = np.where(inf_out, 0.0, np.exp(-alpha * gpu))
    if kind == "winding":
        scale = np.maximum(scale, 1.0)
    err = np.abs(gpu - ref) / scale
    if kind == "smoothdist":  # a non-positive estimate has no distance: +inf matches any oracle estimate <= 0
        err[inf_out & (ref <= 0)] = 0.0
    return err


def rel_error(kind, gpu, ref, alpha=200.0):
    """Plain error against an exact value: relative for Coulomb / affine, relative to max(|F|, 1)
    for winding numbers, and for the smooth distance relative error of the sum exp(-alpha d)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if kind == "smoothdist":
        return np.abs(np.exp(-alpha * gpu) - ref) / ref
    if kind == "winding":
        return np.abs(gpu - ref) / np.maximum(np.abs(ref), 1.0)
    return np.abs(gpu - ref) / np.abs(ref)


def plain_rel_error(gpu, ref):
    """The benchmark spec's tolerance in its stated form: |F_gpu - F_oracle| / |F_oracle| (inf where the
    oracle's estimate is 0)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(ref != 0.0, np.abs(gpu - ref) / np.abs(ref), np.where(gpu == ref, 0.0, np.inf))


def far_from_sources(otree, q):
    """Mask of the queries farther from every source point than the diagonal of that point's own
    leaf cell (the cell of its one-point node in the oracle's 64-ary tree). Next to a source the
    winding kernel's d.N cancels and an FP32 evaluation cannot hold a relative bound. Sources are
    grouped by the level of their cell, and each group is searched for its nearest point."""
    from scipy.spatial import cKDTree
    e = otree.export()
    m = otree.meta()
    pts = otree.points.astype(np.float64)
    leafpt = (e["nchild"] == 0) & (e["end"] - e["begin"] == 1)
    level = np.full(pts.shape[0], -1)
    level[e["perm"][e["begin"][leafpt]]] = e["level"][leafpt]
    qd = np.asarray(q, np.float64)
    ok = np.ones(qd.shape[0], bool)
    for lv in np.unique(level):
        diag = np.inf if lv < 0 else m["diam0"] * np.ldexp(1.0, -2 * int(lv))
        dist, _ = cKDTree(pts[level == lv]).query(qd, k=1)
        ok &= dist > diag
    return ok


def oracle_kwargs(oracle_mod, kind, softening=1e-3, alpha=200.0):
    return dict(kind=KIND_ID[kind], softening=softening, alpha=alpha, affine=AFFINE_G)


def gpu_kwargs(kind, softening=1e-3, alpha=200.0):
    return dict(kernel=kind, softening=softening, alpha=alpha, affine=AFFINE_G)
