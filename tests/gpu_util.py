"""Helpers shared by the GPU parity tests."""
import numpy as np

KIND_ID = {"coulomb": 0, "winding": 1, "smoothdist": 2, "affine": 3}
AFFINE_G = (0.4, -0.3, 0.8)


def dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def parity_error(kind, gpu, ref, alpha=200.0, exact=None):
    """Per-query error of a GPU estimate against the oracle's replay of the same random stream, in
    the units the tolerance uses: relative for Coulomb / affine, relative to max(|F|, 1) for winding
    numbers. For the smooth distance the GPU returns d = -log(F_gpu) / alpha (+inf where its
    estimate of F is <= 0); the error is |F_gpu - F_oracle| / F_exact, the estimate's error relative
    to the exact sum (the estimate itself may cancel to near zero or below), and an output of +inf
    matches an oracle estimate <= 0."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if kind == "smoothdist":
        assert exact is not None, "the smooth-distance error is relative to the exact sum"
        Fg = np.where(np.isposinf(gpu), 0.0, np.exp(-alpha * gpu))
        err = np.abs(Fg - ref) / np.asarray(exact, np.float64)
        err[np.isposinf(gpu) & (ref <= 0)] = 0.0
        return err
    if kind == "winding":
        return np.abs(gpu - ref) / np.maximum(np.abs(ref), 1.0)
    return np.abs(gpu - ref) / np.abs(ref)


def oracle_kwargs(oracle_mod, kind, softening=1e-3, alpha=200.0):
    return dict(kind=KIND_ID[kind], softening=softening, alpha=alpha, affine=AFFINE_G)


def gpu_kwargs(kind, softening=1e-3, alpha=200.0):
    return dict(kernel=kind, softening=softening, alpha=alpha, affine=AFFINE_G)
