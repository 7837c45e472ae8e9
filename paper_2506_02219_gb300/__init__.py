"""Stochastic Barnes-Hut on GB300: Python binding of libsbh.so (include/sbh.h).

Madan, Sharp, Williams, Museth, Levin, "Stochastic Barnes-Hut Approximation for Fast Summation on
the GPU" (SIGGRAPH 2025): the unbiased path estimator of kernel sums F(q) = sum_i m_i f(p_i, q)
that uses the Barnes-Hut level-of-detail hierarchy as a control variate (Sec. 3.3, Algorithm 2).

Every function here only marshals arguments: the work runs in the CUDA kernels of libsbh.so.
There is no CPU fallback; if the library has not been built, loading it raises.

    tree = sbh_build(points, weights, normals=None, leaf_size=1)       # Sec. 3.1, on the GPU
    F    = sbh_eval(tree, queries, kernel="coulomb", samples_per_subdomain=1, seed=0)
    Fbh  = sbh_eval_bh(tree, queries, kernel="coulomb", theta=0.5)      # Algorithm 1
    Fex  = sbh_eval_brute(points, weights, queries, kernel="coulomb")   # Eq. 1

Tensors are float32, contiguous, on the current CUDA device; points and queries are [n, 3].
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = ["SBHError", "Tree", "EvalOpts", "kernel", "load_library", "sbh_build", "sbh_eval", "sbh_eval_count",
           "sbh_eval_bh", "sbh_eval_brute", "sbh_tree_info", "sbh_tree_export", "sbh_tree_free", "sbh_last_error",
           "sbh_version", "sbh_kernel_launches", "sbh_eval_grad", "StochasticSum", "KERNELS", "eval_opts",
           "MultiPlan", "sbh_multi_plan_create", "sbh_multi_plan_launch", "sbh_multi_plan_free"]

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsbh.so")

KERNELS = {"coulomb": 0, "winding": 1, "smoothdist": 2, "affine": 3}
_STATUS = {0: "SBH_OK", 1: "SBH_EINVAL", 2: "SBH_ENOMEM", 3: "SBH_ECUDA", 4: "SBH_ETIMEOUT", 5: "SBH_EUNSUPPORTED"}


class SBHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Kernel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("softening", C.c_float), ("alpha", C.c_float), ("affine", C.c_float * 3)]


class EvalOpts(C.Structure):
    """sbh_eval_opts: sampling (0 mass, 1 count), rr (0 Eq. 5, 1 off, 2 half), seed_mode (0, 1),
    raw_sum (smooth distance: 1 returns the estimated sum instead of the distance), schedule
    (0: warp task batches, 1: one thread per query)."""
    _fields_ = [("sampling", C.c_int32), ("rr", C.c_int32), ("seed_mode", C.c_int32), ("raw_sum", C.c_int32),
                ("schedule", C.c_int32)]


def eval_opts(sampling: int = 0, rr: int = 0, seed_mode: int = 0, raw_sum: int = 0, schedule: int = 0) -> EvalOpts:
    o = EvalOpts()
    o.sampling, o.rr, o.seed_mode, o.raw_sum, o.schedule = sampling, rr, seed_mode, raw_sum, schedule
    return o


class _Meta(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_nodes", C.c_int64), ("leaf_size", C.c_int32),
                ("has_normals", C.c_int32), ("max_depth", C.c_int32), ("reserved", C.c_int32),
                ("first_sub", C.c_int64), ("n_sub", C.c_int64), ("lo", C.c_float * 3), ("side", C.c_float),
                ("diam0", C.c_float), ("reserved_f", C.c_float)]


class _Export(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in ("perm", "code", "begin", "end", "first_child", "nchild", "level",
                                                 "parent", "com_mass", "com_mass64", "dipole", "cdf", "guide")]


_lock = threading.Lock()
_lib = None


def load_library():
    """Load libsbh.so from the package directory; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                               "g.build()'` (there is no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        P, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        lib.sbh_version.restype = i32
        lib.sbh_last_error.restype = C.c_char_p
        lib.sbh_build.argtypes = [P, P, P, i64, i32, P, C.POINTER(P)]
        lib.sbh_eval.argtypes = [P, P, i64, _Kernel, i32, C.c_uint64, C.POINTER(EvalOpts), P, P]
        lib.sbh_eval_count.argtypes = [P, P, i64, _Kernel, i32, C.c_uint64, C.POINTER(EvalOpts), P, P]
        lib.sbh_kernel_launches.restype = C.c_ulonglong
        lib.sbh_eval_grad.argtypes = [P, P, i64, _Kernel, i32, C.c_uint64, C.POINTER(EvalOpts), P, P, P]
        lib.sbh_multi_plan_create.argtypes = [P, P, P, P, i32, _Kernel, i32, C.c_uint64, C.POINTER(EvalOpts), P,
                                              C.POINTER(P)]
        lib.sbh_multi_plan_create.restype = i32
        lib.sbh_multi_plan_launch.argtypes = [P, P]
        lib.sbh_multi_plan_launch.restype = i32
        lib.sbh_multi_plan_free.argtypes = [P]
        lib.sbh_multi_plan_free.restype = None
        lib.sbh_eval_bh.argtypes = [P, P, i64, _Kernel, C.c_float, i32, P, P]
        lib.sbh_eval_brute.argtypes = [P, P, P, i64, P, i64, _Kernel, i32, P, P]
        lib.sbh_eval_brute_grad.argtypes = [P, P, P, i64, P, i64, _Kernel, P, P, P]
        lib.sbh_solve_host.argtypes = [P, P, P, i64, i32, P, i64, _Kernel, i32, C.c_uint64, C.POINTER(EvalOpts),
                                       i64, P, P]
        lib.sbh_solve_host.restype = i32
        lib.sbh_eval_brute_grad.restype = i32
        lib.sbh_tree_info.argtypes = [P, i32, C.POINTER(_Meta)]
        lib.sbh_tree_export.argtypes = [P, i32, C.POINTER(_Export)]
        lib.sbh_tree_free.argtypes = [P]
        lib.sbh_tree_free.restype = None
        lib.sbh_mlp_create.argtypes = [C.c_uint64, P, C.POINTER(P)]
        lib.sbh_mlp_set_weights.argtypes = [P, P, P]
        lib.sbh_mlp_get_weights.argtypes = [P, P, P, P]
        lib.sbh_mlp_scores.argtypes = [P, P, i64, P, P]
        lib.sbh_mlp_get_state.argtypes = [P, P, P, P]
        lib.sbh_mlp_set_state.argtypes = [P, P, i64, P]
        lib.sbh_mlp_loss_grad.argtypes = [P, P, P, P, i64, P, P, P]
        lib.sbh_mlp_dataset.argtypes = [P, P, _Kernel, P, P, P, i64, P, P, P]
        lib.sbh_mlp_train.argtypes = [P, P, P, i64, _Kernel, C.c_float, i32, C.c_float, P, P]
        lib.sbh_eval_learned.argtypes = [P, P, P, i64, _Kernel, i32, C.c_uint64, C.POINTER(EvalOpts), C.c_float, P,
                                         P]
        lib.sbh_set_allocator.argtypes = [P, P, P]
        lib.sbh_set_allocator.restype = i32
        lib.sbh_set_memory_limit.argtypes = [C.c_uint64]
        lib.sbh_set_memory_limit.restype = i32
        lib.sbh_memory_in_use.restype = C.c_uint64
        lib.sbh_mlp_free.argtypes = [P]
        lib.sbh_mlp_free.restype = None
        for f in ("sbh_build", "sbh_eval", "sbh_eval_count", "sbh_eval_grad", "sbh_eval_bh", "sbh_eval_brute",
                  "sbh_tree_info", "sbh_tree_export", "sbh_mlp_create", "sbh_mlp_set_weights",
                  "sbh_mlp_get_weights", "sbh_mlp_get_state", "sbh_mlp_set_state", "sbh_mlp_scores", "sbh_mlp_loss_grad", "sbh_mlp_dataset", "sbh_mlp_train",
                  "sbh_eval_learned"):
            getattr(lib, f).restype = i32
        _lib = lib
        return lib


def _check(status: int):
    if status != 0:
        raise SBHError(status, load_library().sbh_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _dev(t, name, cols=None, allow_none=False):
    """Validate a float32 contiguous CUDA tensor (no silent copies) and return its pointer."""
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous float32")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{name} must have shape [n, {cols}]")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def kernel(kind="coulomb", softening: float = 1e-3, alpha: float = 200.0, affine=(0.0, 0.0, 0.0)) -> _Kernel:
    """sbh_kernel for a kind name ("coulomb", "winding", "smoothdist", "affine") or number."""
    k = _Kernel()
    k.kind = KERNELS[kind] if isinstance(kind, str) else int(kind)
    k.softening = float(softening)
    k.alpha = float(alpha)
    for i in range(3):
        k.affine[i] = float(affine[i])
    return k


class Tree:
    """Owner of an sbh_tree handle; freed with the object (or sbh_tree_free)."""

    def __init__(self, handle: int, n: int, has_normals: bool):
        self._h = C.c_void_p(handle)
        self.n = n
        self.has_normals = has_normals

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            load_library().sbh_tree_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sbh_version() -> int:
    return int(load_library().sbh_version())


def sbh_last_error() -> str:
    return load_library().sbh_last_error().decode(errors="replace")


def sbh_build(points, weights, normals=None, leaf_size: int = 1, stream=None) -> Tree:
    """Build the tree (Sec. 3.1) over points [n, 3], weights [n] (> 0), optional normals [n, 3]."""
    lib = load_library()
    n = int(points.shape[0]) if points is not None else 0
    h = C.c_void_p()
    _check(lib.sbh_build(_dev(points, "points", 3), _dev(weights, "weights"),
                         _dev(normals, "normals", 3, allow_none=True), n, int(leaf_size), _stream(stream),
                         C.byref(h)))
    return Tree(h.value, n, normals is not None)


def _kernel_arg(kind, softening, alpha, affine):
    return kind if isinstance(kind, _Kernel) else kernel(kind, softening, alpha, affine)


def sbh_eval(tree: Tree, queries, kernel="coulomb", samples_per_subdomain: int = 1, seed: int = 0,
             opts: EvalOpts | None = None, out=None, stream=None, softening: float = 1e-3, alpha: float = 200.0,
             affine=(0.0, 0.0, 0.0)):
    """Stochastic estimate (Algorithm 2) at queries [nq, 3]; returns out [nq]."""
    torch = _torch()
    lib = load_library()
    nq = int(queries.shape[0])
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(lib.sbh_eval(tree.handle, _dev(queries, "queries", 3), nq, k, int(samples_per_subdomain),
                        C.c_uint64(int(seed) & (2**64 - 1)), C.byref(opts) if opts is not None else None,
                        _dev(out, "out"), _stream(stream)))
    return out


def sbh_eval_count(tree: Tree, queries, kernel="coulomb", samples_per_subdomain: int = 1, seed: int = 0,
                   opts: EvalOpts | None = None, stream=None, softening: float = 1e-3, alpha: float = 200.0,
                   affine=(0.0, 0.0, 0.0)) -> dict:
    """Work sbh_eval does for these arguments (same paths), counted: kernel terms, node records,
    decisions, prefix fractions read. Synchronises the stream."""
    torch = _torch()
    lib = load_library()
    nq = int(queries.shape[0])
    counts = torch.zeros(4, dtype=torch.int64, device=queries.device)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(lib.sbh_eval_count(tree.handle, _dev(queries, "queries", 3), nq, k, int(samples_per_subdomain),
                              C.c_uint64(int(seed) & (2**64 - 1)), C.byref(opts) if opts is not None else None,
                              C.c_void_p(counts.data_ptr()), _stream(stream)))
    c = counts.cpu().tolist()
    return {"terms": c[0], "records": c[1], "decisions": c[2], "cdf_reads": c[3]}


def sbh_eval_grad(tree: Tree, queries, kernel="coulomb", samples_per_subdomain: int = 1, seed: int = 0,
                  opts: EvalOpts | None = None, out=None, grad=None, stream=None, softening: float = 1e-3,
                  alpha: float = 200.0, affine=(0.0, 0.0, 0.0)):
    """Estimate and its query gradient under the same random stream; returns (out [nq], grad [nq, 3])."""
    torch = _torch()
    lib = load_library()
    nq = int(queries.shape[0])
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    if grad is None:
        grad = torch.empty((nq, 3), dtype=torch.float32, device=queries.device)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(lib.sbh_eval_grad(tree.handle, _dev(queries, "queries", 3), nq, k, int(samples_per_subdomain),
                             C.c_uint64(int(seed) & (2**64 - 1)), C.byref(opts) if opts is not None else None,
                             _dev(out, "out"), _dev(grad, "grad", 3), _stream(stream)))
    return out, grad


def _stochastic_sum_function():
    import torch

    class _StochasticSum(torch.autograd.Function):
        """out = sbh_eval(tree, queries, ...) with backward d out / d queries from sbh_eval_grad (the adjoint
        under the same random stream)."""

        @staticmethod
        def forward(ctx, queries, tree, kernel, samples_per_subdomain, seed, opts, softening, alpha):
            out, grad = sbh_eval_grad(tree, queries.detach().contiguous(), kernel, samples_per_subdomain, seed, opts,
                                      softening=softening, alpha=alpha)
            ctx.save_for_backward(grad)
            return out

        @staticmethod
        def backward(ctx, grad_out):
            (grad,) = ctx.saved_tensors
            return grad_out[:, None] * grad, None, None, None, None, None, None, None

    return _StochasticSum


_SS = None


def StochasticSum(queries, tree: Tree, kernel="coulomb", samples_per_subdomain: int = 1, seed: int = 0,
                  opts: EvalOpts | None = None, softening: float = 1e-3, alpha: float = 200.0):
    """Differentiable estimate: a torch.autograd.Function whose backward is the adjoint traversal."""
    global _SS
    if _SS is None:
        _SS = _stochastic_sum_function()
    return _SS.apply(queries, tree, kernel, samples_per_subdomain, seed, opts, softening, alpha)


class MultiPlan:
    """Owner of an sbh_multi_plan; keeps the trees, queries and outputs it refers to alive."""

    def __init__(self, handle, trees, queries, outs):
        self._h = C.c_void_p(handle)
        self.trees, self.queries, self.outs = list(trees), list(queries), list(outs)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            load_library().sbh_multi_plan_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sbh_multi_plan_create(trees, queries, kernel="coulomb", samples_per_subdomain: int = 1, seed: int = 0,
                          opts: EvalOpts | None = None, outs=None, stream=None, softening: float = 1e-3,
                          alpha: float = 200.0, affine=(0.0, 0.0, 0.0)) -> MultiPlan:
    """A plan that evaluates every (tree, queries) pair in one launch; outputs go to `outs`
    (allocated here if not given, one [nq] tensor per set)."""
    torch = _torch()
    lib = load_library()
    n = len(trees)
    if n != len(queries):
        raise ValueError("one query set per tree")
    if outs is None:
        outs = [torch.empty(int(q.shape[0]), dtype=torch.float32, device=q.device) for q in queries]
    for i, q in enumerate(queries):
        if q.shape[0] > 0:
            _dev(q, f"queries[{i}]", 3)
            _dev(outs[i], f"outs[{i}]")
    th = (C.c_void_p * n)(*[t.handle.value for t in trees])
    qh = (C.c_void_p * n)(*[q.data_ptr() if q.shape[0] > 0 else 0 for q in queries])
    oh = (C.c_void_p * n)(*[o.data_ptr() if o.shape[0] > 0 else 0 for o in outs])
    nq = (C.c_int64 * n)(*[int(q.shape[0]) for q in queries])
    k = _kernel_arg(kernel, softening, alpha, affine)
    h = C.c_void_p()
    _check(lib.sbh_multi_plan_create(C.cast(th, C.c_void_p), C.cast(qh, C.c_void_p), C.cast(nq, C.c_void_p),
                                     C.cast(oh, C.c_void_p), n, k, int(samples_per_subdomain),
                                     C.c_uint64(int(seed) & (2**64 - 1)), C.byref(opts) if opts is not None else None,
                                     _stream(stream), C.byref(h)))
    return MultiPlan(h.value, trees, queries, outs)


def sbh_multi_plan_launch(plan: MultiPlan, stream=None):
    """Run every set of the plan in one launch (capturable in a CUDA graph); returns the outputs."""
    _check(load_library().sbh_multi_plan_launch(plan.handle, _stream(stream)))
    return plan.outs


def sbh_multi_plan_free(plan: MultiPlan) -> None:
    plan.free()


def capture_multi(plan: MultiPlan):
    """Capture one launch of the plan into a torch.cuda.CUDAGraph; graph.replay() re-runs it.
    graph.sbh_kernels is the number of the library's kernels one replay launches."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside the capture
        sbh_multi_plan_launch(plan)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    n0 = sbh_kernel_launches()
    with torch.cuda.graph(g):
        sbh_multi_plan_launch(plan)
    g.sbh_kernels = sbh_kernel_launches() - n0
    return g


def sbh_kernel_launches() -> int:
    """CUDA kernels launched by libsbh.so in this process so far."""
    return int(load_library().sbh_kernel_launches())


def sbh_eval_bh(tree: Tree, queries, kernel="coulomb", theta: float = 0.5, warp_vote: bool = True, out=None,
                stream=None, softening: float = 1e-3, alpha: float = 200.0, affine=(0.0, 0.0, 0.0)):
    """Deterministic Barnes-Hut (Algorithm 1) with beta = 1 / theta; returns out [nq]."""
    torch = _torch()
    lib = load_library()
    nq = int(queries.shape[0])
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(lib.sbh_eval_bh(tree.handle, _dev(queries, "queries", 3), nq, k, C.c_float(theta), int(bool(warp_vote)),
                           _dev(out, "out"), _stream(stream)))
    return out


def sbh_eval_brute(points, weights, queries, kernel="coulomb", normals=None, fp64_accum: bool = True, out=None,
                   stream=None, softening: float = 1e-3, alpha: float = 200.0, affine=(0.0, 0.0, 0.0)):
    """Exact sum (Eq. 1) by tiled brute force; returns out [nq]."""
    torch = _torch()
    lib = load_library()
    nq = int(queries.shape[0])
    n = int(points.shape[0])
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(lib.sbh_eval_brute(_dev(points, "points", 3), _dev(weights, "weights"),
                              _dev(normals, "normals", 3, allow_none=True), n, _dev(queries, "queries", 3), nq, k,
                              int(bool(fp64_accum)), _dev(out, "out"), _stream(stream)))
    return out


def _host(a, name, cols=None, allow_none=False):
    """Pointer to a contiguous float32 host buffer (numpy array or CPU tensor, pinned or not)."""
    import numpy as np
    if a is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 CPU tensor")
        ptr, shape = a.data_ptr(), tuple(a.shape)
    else:
        if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
            raise ValueError(f"{name} must be a C-contiguous float32 numpy array")
        ptr, shape = a.ctypes.data, a.shape
    if cols is not None and (len(shape) != 2 or shape[1] != cols):
        raise ValueError(f"{name} must have shape [n, {cols}]")
    return C.c_void_p(ptr)


def sbh_solve_host(points, weights, queries, normals=None, leaf_size: int = 1, kernel="coulomb",
                   samples_per_subdomain: int = 1, seed: int = 0, opts: EvalOpts | None = None, chunk: int = 0,
                   out=None, stream=None, softening: float = 1e-3, alpha: float = 200.0, affine=(0.0, 0.0, 0.0)):
    """One-shot build and evaluation from host buffers (numpy arrays or CPU tensors; page-locked
    memory lets the copies overlap the work); returns out (host, float32 [nq])."""
    import numpy as np
    n, nq = int(points.shape[0]), int(queries.shape[0])
    if out is None:
        out = np.empty(nq, dtype=np.float32)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(load_library().sbh_solve_host(_host(points, "points", 3), _host(weights, "weights"),
                                         _host(normals, "normals", 3, allow_none=True), n, int(leaf_size),
                                         _host(queries, "queries", 3), nq, k, int(samples_per_subdomain),
                                         C.c_uint64(int(seed) & (2**64 - 1)),
                                         C.byref(opts) if opts is not None else None, int(chunk),
                                         _host(out, "out"), _stream(stream)))
    return out


def sbh_eval_brute_grad(points, weights, queries, kernel="coulomb", normals=None, out=None, grad=None, stream=None,
                        softening: float = 1e-3, alpha: float = 200.0, affine=(0.0, 0.0, 0.0)):
    """Exact sum and its query gradient by tiled brute force (FP64 accumulation), in the
    conventions of sbh_eval_grad; returns (out [nq], grad [nq, 3])."""
    torch = _torch()
    n, nq = int(points.shape[0]), int(queries.shape[0])
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    if grad is None:
        grad = torch.empty((nq, 3), dtype=torch.float32, device=queries.device)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(load_library().sbh_eval_brute_grad(_dev(points, "points", 3), _dev(weights, "weights"),
                                              _dev(normals, "normals", 3, allow_none=True), n,
                                              _dev(queries, "queries", 3), nq, k, _dev(out, "out"),
                                              _dev(grad, "grad", 3), _stream(stream)))
    return out, grad


def sbh_tree_info(tree: Tree, which: int = 0) -> dict:
    m = _Meta()
    _check(load_library().sbh_tree_info(tree.handle, int(which), C.byref(m)))
    return {"n_points": m.n_points, "n_nodes": m.n_nodes, "leaf_size": m.leaf_size, "has_normals": bool(m.has_normals),
            "max_depth": m.max_depth, "first_sub": m.first_sub, "n_sub": m.n_sub, "lo": np.array(m.lo[:], np.float32),
            "side": m.side, "diam0": m.diam0}


def sbh_tree_export(tree: Tree, which: int = 0) -> dict:
    """Host copy of a tree: numpy arrays keyed like sbh_tree_export_buffers."""
    info = sbh_tree_info(tree, which)
    n, N = info["n_points"], info["n_nodes"]
    a = {"perm": np.zeros(n, np.int32), "code": np.zeros(n, np.uint64), "begin": np.zeros(N, np.int32),
         "end": np.zeros(N, np.int32), "first_child": np.zeros(N, np.int32), "nchild": np.zeros(N, np.int32),
         "level": np.zeros(N, np.int32), "parent": np.zeros(N, np.int32), "com_mass": np.zeros((N, 4), np.float32),
         "com_mass64": np.zeros((N, 4), np.float64), "dipole": np.zeros((N, 3), np.float32),
         "cdf": np.zeros(N, np.float32), "guide": np.zeros(N, np.uint8)}
    e = _Export()
    for name, arr in a.items():
        setattr(e, name, arr.ctypes.data_as(C.c_void_p))
    _check(load_library().sbh_tree_export(tree.handle, int(which), C.byref(e)))
    a["info"] = info
    return a


def sbh_tree_free(tree: Tree) -> None:
    tree.free()


MLP_PARAMS = 1313


class Mlp:
    """Owner of an sbh_mlp handle (the learned child proposal); freed with the object."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            load_library().sbh_mlp_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sbh_mlp_create(seed: int = 0, stream=None) -> Mlp:
    """New 6-32-32-1 proposal network with weights drawn from `seed`."""
    lib = load_library()
    h = C.c_void_p()
    _check(lib.sbh_mlp_create(C.c_uint64(int(seed) & (2**64 - 1)), _stream(stream), C.byref(h)))
    return Mlp(h.value)


def sbh_mlp_set_weights(net: Mlp, weights, stream=None) -> None:
    """Load FP32 master weights (any array-like of MLP_PARAMS values)."""
    import numpy as np
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).reshape(-1))
    if w.size != MLP_PARAMS:
        raise ValueError(f"weights must hold {MLP_PARAMS} values")
    _check(load_library().sbh_mlp_set_weights(net.handle, w.ctypes.data_as(C.c_void_p), _stream(stream)))


def sbh_mlp_get_weights(net: Mlp, stream=None):
    """Return (FP32 master weights as numpy [MLP_PARAMS], Adam steps taken)."""
    import numpy as np
    w = np.empty(MLP_PARAMS, dtype=np.float32)
    step = C.c_int64(0)
    _check(load_library().sbh_mlp_get_weights(net.handle, w.ctypes.data_as(C.c_void_p), C.byref(step),
                                              _stream(stream)))
    return w, int(step.value)


def sbh_mlp_get_state(net: Mlp, stream=None) -> dict:
    """Training state for a checkpoint: {"weights", "adam_m", "adam_v"} (numpy FP32) and "adam_step"."""
    import numpy as np
    st = np.empty(3 * MLP_PARAMS, dtype=np.float32)
    step = C.c_int64(0)
    _check(load_library().sbh_mlp_get_state(net.handle, st.ctypes.data_as(C.c_void_p), C.byref(step),
                                            _stream(stream)))
    return {"weights": st[:MLP_PARAMS].copy(), "adam_m": st[MLP_PARAMS:2 * MLP_PARAMS].copy(),
            "adam_v": st[2 * MLP_PARAMS:].copy(), "adam_step": int(step.value)}


def sbh_mlp_set_state(net: Mlp, state: dict, stream=None) -> None:
    """Restore a state from sbh_mlp_get_state."""
    import numpy as np
    st = np.ascontiguousarray(np.concatenate([np.asarray(state[k], np.float32).reshape(-1)
                                              for k in ("weights", "adam_m", "adam_v")]))
    if st.size != 3 * MLP_PARAMS:
        raise ValueError("state arrays must hold MLP_PARAMS values each")
    _check(load_library().sbh_mlp_set_state(net.handle, st.ctypes.data_as(C.c_void_p), int(state["adam_step"]),
                                            _stream(stream)))


def save_mlp(net: Mlp, path: str) -> None:
    """Write the training state to an .npz checkpoint."""
    import numpy as np
    np.savez(path, **sbh_mlp_get_state(net))


def load_mlp(path: str, stream=None) -> Mlp:
    """A network restored from an .npz checkpoint written by save_mlp."""
    import numpy as np
    with np.load(path) as z:
        state = {k: z[k] for k in ("weights", "adam_m", "adam_v")}
        state["adam_step"] = int(z["adam_step"])
    net = sbh_mlp_create(0, stream)
    sbh_mlp_set_state(net, state, stream)
    return net


def sbh_mlp_scores(net: Mlp, feats, out=None, stream=None):
    """Scores of feature rows [n, 6] with the FP16 inference weights; returns [n]."""
    torch = _torch()
    n = int(feats.shape[0])
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=feats.device)
    _check(load_library().sbh_mlp_scores(net.handle, _dev(feats, "feats", 6), n, _dev(out, "out"), _stream(stream)))
    return out


def sbh_mlp_loss_grad(net: Mlp, feats, targets, offsets, stream=None):
    """Mean set cross-entropy and its gradient in the master weights; returns (loss [1], grad [MLP_PARAMS])."""
    torch = _torch()
    if not (isinstance(offsets, torch.Tensor) and offsets.is_cuda and offsets.dtype == torch.int64
            and offsets.is_contiguous()):
        raise ValueError("offsets must be a contiguous int64 CUDA tensor")
    n_sets = int(offsets.numel()) - 1
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=feats.device)
    loss = torch.empty(1, dtype=torch.float32, device=feats.device)
    _check(load_library().sbh_mlp_loss_grad(net.handle, _dev(feats, "feats", 6), _dev(targets, "targets"),
                                            C.c_void_p(offsets.data_ptr()), n_sets, _dev(grad, "grad"),
                                            _dev(loss, "loss"), _stream(stream)))
    return loss, grad


def _int_dev(t, name, dtype):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
    return C.c_void_p(t.data_ptr())


def sbh_mlp_dataset(tree: Tree, queries, set_query, set_node, set_offsets, kernel="coulomb", stream=None,
                    softening: float = 1e-3, alpha: float = 200.0, affine=(0.0, 0.0, 0.0)):
    """Features [rows, 6] and |exact child residual| targets [rows] of explicit decision sets
    (node set_node[s] at query set_query[s], int32; rows set_offsets[s] .. set_offsets[s+1]-1, int64)."""
    torch = _torch()
    torch_i32, torch_i64 = torch.int32, torch.int64
    n_sets = int(set_node.numel())
    rows = int(set_offsets[-1].item()) if n_sets else 0
    feats = torch.empty((rows, 6), dtype=torch.float32, device=queries.device)
    targets = torch.empty(rows, dtype=torch.float32, device=queries.device)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(load_library().sbh_mlp_dataset(tree.handle, _dev(queries, "queries", 3), k,
                                          _int_dev(set_query, "set_query", torch_i32),
                                          _int_dev(set_node, "set_node", torch_i32),
                                          _int_dev(set_offsets, "set_offsets", torch_i64), n_sets,
                                          _dev(feats, "feats", 6), _dev(targets, "targets"), _stream(stream)))
    return feats, targets


def sbh_mlp_train(net: Mlp, tree: Tree, queries, kernel="coulomb", near: float = float("inf"), steps: int = 200,
                  lr: float = 3e-3, stream=None, softening: float = 1e-3, alpha: float = 200.0,
                  affine=(0.0, 0.0, 0.0)):
    """Fit the proposal to the residuals at the decisions the estimator's own paths reach from the
    training queries [nq, 3]; returns the loss before each step (numpy [steps])."""
    import numpy as np
    losses = np.zeros(max(int(steps), 1), dtype=np.float32)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(load_library().sbh_mlp_train(net.handle, tree.handle, _dev(queries, "queries", 3), int(queries.shape[0]),
                                        k, C.c_float(near), int(steps), C.c_float(lr),
                                        losses.ctypes.data_as(C.c_void_p), _stream(stream)))
    return losses[:int(steps)]


def sbh_eval_learned(tree: Tree, net: Mlp, queries, kernel="coulomb", samples_per_subdomain: int = 1,
                     seed: int = 0, opts: EvalOpts | None = None, near: float = float("inf"), out=None, stream=None,
                     softening: float = 1e-3, alpha: float = 200.0, affine=(0.0, 0.0, 0.0)):
    """Estimate with the learned child proposal at nodes nearer than `near` cell diagonals; returns out [nq]."""
    torch = _torch()
    nq = int(queries.shape[0])
    if out is None:
        out = torch.empty(nq, dtype=torch.float32, device=queries.device)
    k = _kernel_arg(kernel, softening, alpha, affine)
    _check(load_library().sbh_eval_learned(tree.handle, net.handle, _dev(queries, "queries", 3), nq, k,
                                           int(samples_per_subdomain), C.c_uint64(int(seed) & (2**64 - 1)),
                                           C.byref(opts) if opts is not None else None, C.c_float(near),
                                           _dev(out, "out"), _stream(stream)))
    return out


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_allocator_keepalive = None


def sbh_set_allocator(alloc=None, free=None) -> None:
    """Route the library's device memory through alloc(bytes, stream_handle) -> int pointer and
    free(ptr, stream_handle); None, None restores the library's own pool."""
    global _allocator_keepalive
    lib = load_library()
    if (alloc is None) != (free is None):
        raise ValueError("give both allocator functions or neither")
    if alloc is None:
        _check(lib.sbh_set_allocator(None, None, None))
        _allocator_keepalive = None
        return

    def _a(nbytes, stream, ctx):
        try:
            return int(alloc(int(nbytes), stream or 0)) or None
        except Exception:
            return None

    def _f(ptr, stream, ctx):
        free(int(ptr), stream or 0)

    cbs = (ALLOC_FN(_a), FREE_FN(_f))
    _check(lib.sbh_set_allocator(C.cast(cbs[0], C.c_void_p), C.cast(cbs[1], C.c_void_p), None))
    _allocator_keepalive = cbs


def use_torch_allocator() -> None:
    """Take the library's device memory from PyTorch's caching allocator (stream-ordered on the
    stream of each library call)."""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    sbh_set_allocator(alloc, free)


def sbh_set_memory_limit(nbytes: int) -> None:
    """Cap the device bytes the library holds at once (0: no cap); beyond it calls fail with SBH_ENOMEM."""
    _check(load_library().sbh_set_memory_limit(C.c_uint64(int(nbytes))))


def sbh_memory_in_use() -> int:
    return int(load_library().sbh_memory_in_use())
