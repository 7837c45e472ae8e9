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


def oracle_kwargs(oracle_mod, kind, softening=1e-3, alpha=200.0):
    return dict(kind=KIND_ID[kind], softening=softening, alpha=alpha, affine=AFFINE_G)


def gpu_kwargs(kind, softening=1e-3, alpha=200.0):
    return dict(kernel=kind, softening=softening, alpha=alpha, affine=AFFINE_G)
