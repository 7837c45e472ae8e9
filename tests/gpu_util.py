"""Helpers shared by the GPU parity tests."""
import numpy as np

KIND_ID = {"coulomb": 0, "winding": 1, "smoothdist": 2, "affine": 3}
AFFINE_G = (0.4, -0.3, 0.8)


def dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def parity_error(kind, gpu, ref, alpha=200.0):
    """Per-query error of a GPU estimate against an oracle value, in the units the tolerance uses:
    relative for Coulomb / affine, relative to max(|F|, 1) for winding numbers, and for the smooth
    distance the difference of log F (= alpha * distance), i.e. the relative error of the sum."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if kind == "smoothdist":
        # gpu is -log(F_gpu)/alpha, +inf where the estimate of F is <= 0
        err = np.full(ref.shape, np.inf)
        pos = ref > 0
        err[pos] = np.abs(alpha * gpu[pos] + np.log(ref[pos]))
        err[~pos & np.isposinf(gpu)] = 0.0
        return err
    if kind == "winding":
        return np.abs(gpu - ref) / np.maximum(np.abs(ref), 1.0)
    return np.abs(gpu - ref) / np.abs(ref)


def oracle_kwargs(oracle_mod, kind, softening=1e-3, alpha=200.0):
    return dict(kind=KIND_ID[kind], softening=softening, alpha=alpha, affine=AFFINE_G)


def gpu_kwargs(kind, softening=1e-3, alpha=200.0):
    return dict(kernel=kind, softening=softening, alpha=alpha, affine=AFFINE_G)
