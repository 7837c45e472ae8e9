"""FP64 CPU oracle for the stochastic Barnes-Hut hot path (Madan et al., SIGGRAPH 2025).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg import this package. The CUDA library never does, and this package imports nothing
from it: the two are independent restatements of the paper.

The arithmetic lives in ``sbh_oracle.c`` (plain C, FP64 sums, FP32 decisions, OpenMP over
queries); this module compiles it with the host C compiler and marshals numpy arrays.

Functions and the passages they follow:
  brute(...)        Eq. 1, the exact kernel sum.
  Tree(...)         Sec. 3.1, the octree-like tree with aggregate mass and centre of mass. The
                    options box=, collapse= and subdomain_generation= select alternative readings
                    of Sec. 3.1 and Sec. 3.3.1 (oracle only; the CUDA path implements the default).
  Tree.bh(...)      Algorithm 1 (Barnes-Hut), Eq. 2; Tree.bh_work counts its node tests and terms.
  Tree.replay(...)  Algorithm 2 with Eq. 5 (Russian roulette), Eq. 6 (swap), Eq. 7 (estimator),
                    driven by the same counter-based Philox4x32-10 stream as the GPU kernel.
  Tree.enumerate()  exact mean and variance of Eq. 7 by enumeration (Appendix A).
  brute_grad, Tree.replay_grad, Tree.enumerate_grad: the same for the query gradient (the
                    estimator applied to grad_q f with the paths and weights held fixed).
  philox(...)       Philox4x32-10 (Salmon et al., SC'11).

Parity pins (tests/test_oracle_*.py): closed forms for the brute force, hand-built trees,
enumeration == brute force (the theorem), zero variance for an affine kernel, replay statistics
against the enumerated distribution, Philox against an independent implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbh_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

COULOMB, WINDING, SMOOTHDIST, AFFINE = 0, 1, 2, 3
SAMPLE_MASS, SAMPLE_COUNT = 0, 1
RR_PAPER, RR_OFF, RR_HALF = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile sbh_oracle.c into liboracle.so next to it (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Kernel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("softening", C.c_double), ("alpha", C.c_double),
                ("affine", C.c_double * 3)]


class _Opts(C.Structure):
    _fields_ = [("sampling", C.c_int32), ("rr", C.c_int32), ("coherent", C.c_int32),
                ("abs_mode", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # SBHO_LIB: load a separately built copy (the sanitizer test builds one with ASan/UBSan)
        lib = C.CDLL(os.environ.get("SBHO_LIB") or build())
        P = C.c_void_p
        i64, i32, u64 = C.c_int64, C.c_int32, C.c_uint64
        lib.sbho_philox4x32_10.argtypes = [P, P, P]
        lib.sbho_brute.argtypes = [C.POINTER(_Kernel), P, P, P, i64, P, i64, P]
        lib.sbho_tree_build.argtypes = [P, P, P, i64, i32, i32]
        lib.sbho_tree_build.restype = P
        lib.sbho_tree_build_ex.argtypes = [P, P, P, i64, i32, i32, i32, i32, i32]
        lib.sbho_tree_build_ex.restype = P
        lib.sbho_bh_work.argtypes = [P, P, i64, C.c_float, P]
        lib.sbho_replay_cut.argtypes = [P, C.POINTER(_Kernel), P, i64, C.c_float, u64, P, P]
        lib.sbho_enumerate_cut.argtypes = [P, C.POINTER(_Kernel), P, i64, C.c_float, P, P]
        lib.sbho_tree_free.argtypes = [P]
        lib.sbho_tree_nnodes.argtypes = [P]
        lib.sbho_tree_nnodes.restype = i64
        lib.sbho_tree_meta.argtypes = [P, P, P]
        lib.sbho_tree_export.argtypes = [P] + [P] * 11
        lib.sbho_bh.argtypes = [P, C.POINTER(_Kernel), P, i64, C.c_float, P]
        lib.sbho_replay.argtypes = [P, C.POINTER(_Kernel), P, i64, i32, u64, C.POINTER(_Opts), P, P, P, P, P]
        lib.sbho_enumerate.argtypes = [P, C.POINTER(_Kernel), P, i64, C.POINTER(_Opts), P, P]
        lib.sbho_brute_grad.argtypes = [C.POINTER(_Kernel), P, P, P, i64, P, i64, P]
        lib.sbho_replay_grad.argtypes = [P, C.POINTER(_Kernel), P, P, i64, i32, u64, C.POINTER(_Opts), P, P, P, P]
        lib.sbho_enumerate_grad.argtypes = [P, C.POINTER(_Kernel), P, i64, C.POINTER(_Opts), P]
        lib.sbho_mlp_nparam.restype = i32
        lib.sbho_mlp_forward.argtypes = [P, P, i64, P]
        lib.sbho_mlp_loss_grad.argtypes = [P, P, P, P, i64, P]
        lib.sbho_mlp_loss_grad.restype = C.c_double
        lib.sbho_child_features.argtypes = [P, i64, P, i32, P]
        lib.sbho_enumerate_learned.argtypes = [P, C.POINTER(_Kernel), P, C.c_double, C.c_float, P, i64, P, P]
        lib.sbho_max_threads.restype = i32
        lib.sbho_set_threads.argtypes = [i32]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a, cols=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def kernel(kind: int, softening: float = 1e-3, alpha: float = 200.0, affine=(0.0, 0.0, 0.0)) -> _Kernel:
    k = _Kernel()
    k.kind = int(kind)
    k.softening = float(softening)
    k.alpha = float(alpha)
    for i in range(3):
        k.affine[i] = float(affine[i])
    return k


def _opts(sampling=SAMPLE_MASS, rr=RR_PAPER, coherent=False, abs_mode=0) -> _Opts:
    o = _Opts()
    o.sampling, o.rr, o.coherent, o.abs_mode = int(sampling), int(rr), int(bool(coherent)), int(abs_mode)
    return o


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter block (4 x u32) under a key (2 x u32)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib.sbho_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def brute(points, weights, queries, kind=COULOMB, normals=None, softening=1e-3, alpha=200.0,
          affine=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Eq. 1: F(q) = sum_i m_i f(p_i, q), FP64 with compensated summation. For the smooth
    distance kernel this is the sum of exponentials (take -log(F)/alpha for the distance)."""
    lib = _load()
    pts, w, q = _f32(points, 3), _f32(weights), _f32(queries, 3)
    nrm = _f32(normals, 3)
    out = np.zeros(q.shape[0], dtype=np.float64)
    k = kernel(kind, softening, alpha, affine)
    lib.sbho_brute(C.byref(k), _ptr(pts), _ptr(w), _ptr(nrm), pts.shape[0], _ptr(q), q.shape[0], _ptr(out))
    return out


def brute_grad(points, weights, queries, kind=COULOMB, normals=None, softening=1e-3, alpha=200.0,
               affine=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Gradient of Eq. 1 with respect to the query position, [nq, 3], FP64 compensated sums."""
    lib = _load()
    pts, w, q = _f32(points, 3), _f32(weights), _f32(queries, 3)
    nrm = _f32(normals, 3)
    out = np.zeros((q.shape[0], 3), dtype=np.float64)
    k = kernel(kind, softening, alpha, affine)
    lib.sbho_brute_grad(C.byref(k), _ptr(pts), _ptr(w), _ptr(nrm), pts.shape[0], _ptr(q), q.shape[0], _ptr(out))
    return out


BOX_MODES = {"cell": 0, "tight": 1, "tight_literal": 2}


class Tree:
    """The oracle's tree over (points, weights[, normals]) with per-dimension branching d.

    The defaults are the readings the CUDA path implements. The other settings exist in the
    oracle alone, to measure what each reading of the paper does to the estimator:
      box="cell"           |B_a| = diagonal of the node's octree cell (default)
      box="tight"          |B_a| = diagonal of the tight box of the node's points (Sec. 3.1's
                           wording); a node of zero extent takes its cell's diagonal
      box="tight_literal"  the tight box everywhere: Eq. 5 gives p = 0 into one-point nodes, so
                           the estimator never takes the swaps above them (it is truncated)
      collapse=False       single-child chains are kept as nodes (default: they collapse)
      subdomain_generation=g  subdomains are the nodes g generations below the root, plus any
                           leaf above that (default 1: the root's children, Sec. 3.3.1)
    """

    def __init__(self, points, weights, normals=None, leaf_size: int = 1, d: int = 4, box: str = "cell",
                 collapse: bool = True, subdomain_generation: int = 1):
        lib = _load()
        self.points = _f32(points, 3)
        self.weights = _f32(weights)
        self.normals = _f32(normals, 3)
        self.n = self.points.shape[0]
        self.d = d
        if box not in BOX_MODES:
            raise ValueError(f"box must be one of {sorted(BOX_MODES)}")
        h = lib.sbho_tree_build_ex(_ptr(self.points), _ptr(self.weights), _ptr(self.normals), self.n,
                                   int(leaf_size), int(d), BOX_MODES[box], int(bool(collapse)),
                                   int(subdomain_generation))
        if not h:
            raise ValueError("oracle tree build rejected its inputs")
        self._h = h
        self._lib = lib
        self.n_nodes = int(lib.sbho_tree_nnodes(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.sbho_tree_free(h)
            self._h = None

    def meta(self) -> dict:
        m = np.zeros(5, dtype=np.float32)
        ids = np.zeros(2, dtype=np.int64)
        self._lib.sbho_tree_meta(self._h, _ptr(m), _ptr(ids))
        return {"lo": m[:3].copy(), "side": float(m[3]), "diam0": float(m[4]),
                "first_sub": int(ids[0]), "n_sub": int(ids[1])}

    def export(self) -> dict:
        n, N = self.n, self.n_nodes
        a = {
            "perm": np.zeros(n, np.int64), "code": np.zeros(n, np.uint64),
            "begin": np.zeros(N, np.int64), "end": np.zeros(N, np.int64),
            "first_child": np.zeros(N, np.int64), "nchild": np.zeros(N, np.int32),
            "level": np.zeros(N, np.int32), "mass": np.zeros(N, np.float64),
            "com": np.zeros((N, 3), np.float64), "dip": np.zeros((N, 3), np.float64),
            "cdf": np.zeros(N, np.float32),
        }
        self._lib.sbho_tree_export(self._h, *[_ptr(a[k]) for k in
                                              ("perm", "code", "begin", "end", "first_child", "nchild",
                                               "level", "mass", "com", "dip", "cdf")])
        return a

    def bh(self, queries, beta: float, kind=COULOMB, softening=1e-3, alpha=200.0,
           affine=(0.0, 0.0, 0.0)) -> np.ndarray:
        """Algorithm 1 for every query; beta = inf gives the exact sum."""
        q = _f32(queries, 3)
        out = np.zeros(q.shape[0], np.float64)
        k = kernel(kind, softening, alpha, affine)
        self._lib.sbho_bh(self._h, C.byref(k), _ptr(q), q.shape[0], C.c_float(beta), _ptr(out))
        return out

    def bh_work(self, queries, beta: float) -> np.ndarray:
        """Algorithm 1's work per query: far-field tests of the nodes it opens plus the terms it
        adds (int64)."""
        q = _f32(queries, 3)
        out = np.zeros(q.shape[0], np.int64)
        self._lib.sbho_bh_work(self._h, _ptr(q), q.shape[0], C.c_float(beta), _ptr(out))
        return out

    def replay(self, queries, S: int = 1, seed: int = 0, kind=COULOMB, softening=1e-3, alpha=200.0,
               affine=(0.0, 0.0, 0.0), sampling=SAMPLE_MASS, rr=RR_PAPER, coherent=False,
               return_swaps=False, query_index=None, return_abs_sum=False, abs_mode=0, return_terms=False):
        """Algorithm 2 replayed with the Philox stream; returns the FP64 estimate of the kernel
        sum per query (the sum of exponentials for the smooth distance kernel). query_index gives
        each query's index in the random stream (default: its position). With return_abs_sum the
        sum of the absolute values of all terms the estimate adds is returned too (the scale of
        the rounding error of any evaluation of the same signed sum). abs_mode=1 sums instead, for
        the winding kernel, each term's sensitivity to rounding its node record to FP32,
        |N| (r + 4 |p|) / (4 pi r^3): the scale that applies where d.N cancels, next to the surface.
        return_terms adds the number of kernel terms evaluated per query (control variates plus
        every swap's children and node)."""
        q = _f32(queries, 3)
        qidx = None if query_index is None else np.ascontiguousarray(np.asarray(query_index, dtype=np.uint32))
        out = np.zeros(q.shape[0], np.float64)
        swaps = np.zeros(q.shape[0], np.int64)
        k = kernel(kind, softening, alpha, affine)
        o = _opts(sampling, rr, coherent, abs_mode)
        absum = np.zeros(q.shape[0], np.float64)
        terms = np.zeros(q.shape[0], np.int64)
        self._lib.sbho_replay(self._h, C.byref(k), _ptr(q), q.shape[0], int(S), C.c_uint64(seed & (2**64 - 1)),
                              C.byref(o), _ptr(qidx), _ptr(out), _ptr(swaps), _ptr(absum), _ptr(terms))
        res = (out,)
        if return_swaps:
            res += (swaps,)
        if return_abs_sum:
            res += (absum,)
        if return_terms:
            res += (terms,)
        return res if len(res) > 1 else out

    def replay_grad(self, queries, S: int = 1, seed: int = 0, kind=COULOMB, softening=1e-3, alpha=200.0,
                    affine=(0.0, 0.0, 0.0), sampling=SAMPLE_MASS, rr=RR_PAPER, coherent=False, query_index=None,
                    eval_at=None):
        """The estimator with paths and weights drawn at `queries` (FP32 decisions, as replay) and every
        term replaced by its query gradient evaluated at `eval_at` (default: the same queries, FP64).
        Returns (value estimate along those paths at eval_at [nq], gradient [nq, 3], sum of |gradient
        terms| [nq])."""
        q = _f32(queries, 3)
        qv = np.ascontiguousarray(q.astype(np.float64) if eval_at is None else np.asarray(eval_at, np.float64)
                                  .reshape(-1, 3))
        qidx = None if query_index is None else np.ascontiguousarray(np.asarray(query_index, dtype=np.uint32))
        val = np.zeros(q.shape[0], np.float64)
        grad = np.zeros((q.shape[0], 3), np.float64)
        ab = np.zeros(q.shape[0], np.float64)
        k = kernel(kind, softening, alpha, affine)
        o = _opts(sampling, rr, coherent)
        self._lib.sbho_replay_grad(self._h, C.byref(k), _ptr(q), _ptr(qv), q.shape[0], int(S),
                                   C.c_uint64(seed & (2**64 - 1)), C.byref(o), _ptr(qidx), _ptr(val), _ptr(grad),
                                   _ptr(ab))
        return val, grad, ab

    def enumerate_grad(self, queries, kind=COULOMB, softening=1e-3, alpha=200.0, affine=(0.0, 0.0, 0.0),
                       sampling=SAMPLE_MASS, rr=RR_PAPER):
        """Exact mean of the one-sample gradient estimator per query, [nq, 3], by enumeration."""
        q = _f32(queries, 3)
        mean = np.zeros((q.shape[0], 3), np.float64)
        k = kernel(kind, softening, alpha, affine)
        o = _opts(sampling, rr, False)
        self._lib.sbho_enumerate_grad(self._h, C.byref(k), _ptr(q), q.shape[0], C.byref(o), _ptr(mean))
        return mean

    def child_features(self, node: int, query, use_dipole: bool = False) -> np.ndarray:
        """Learned-proposal features [nchild, 6] of the children of `node` at `query` (FP64)."""
        e = self.export()
        nc = int(e["nchild"][node])
        x = np.zeros((nc, 6), np.float64)
        q = _f32(np.asarray(query).reshape(1, 3), 3)
        self._lib.sbho_child_features(self._h, int(node), _ptr(q), int(bool(use_dipole)), _ptr(x))
        return x

    def enumerate_learned(self, queries, weights, eps: float = 0.1, kind=COULOMB, softening=1e-3, alpha=200.0,
                          affine=(0.0, 0.0, 0.0), near: float = float("inf")):
        """Exact (mean, variance) of the one-sample estimator with the learned proposal, used at
        nodes with at most 64 children nearer to the query than `near` cell diagonals."""
        q = _f32(queries, 3)
        w = np.ascontiguousarray(np.asarray(weights, np.float64))
        mean = np.zeros(q.shape[0], np.float64)
        var = np.zeros(q.shape[0], np.float64)
        k = kernel(kind, softening, alpha, affine)
        self._lib.sbho_enumerate_learned(self._h, C.byref(k), _ptr(w), C.c_double(eps), C.c_float(near), _ptr(q),
                                         q.shape[0],
                                         _ptr(mean), _ptr(var))
        return mean, var

    def replay_cut(self, queries, beta_s: float, seed: int = 0, kind=COULOMB, softening=1e-3, alpha=200.0,
                   affine=(0.0, 0.0, 0.0)):
        """The estimator with per-query subdomains taken as the Barnes-Hut contribution nodes at beta_s
        (the alternative cover Sec. 3.3.1 names), S = 1, mass p_agg, Eq. 5 roulette. Returns (estimate,
        work per query: the walk's far-field tests plus every swap's children and node)."""
        q = _f32(queries, 3)
        out = np.zeros(q.shape[0], np.float64)
        work = np.zeros(q.shape[0], np.int64)
        k = kernel(kind, softening, alpha, affine)
        self._lib.sbho_replay_cut(self._h, C.byref(k), _ptr(q), q.shape[0], C.c_float(beta_s),
                                  C.c_uint64(seed & (2**64 - 1)), _ptr(out), _ptr(work))
        return out, work

    def enumerate_cut(self, queries, beta_s: float, kind=COULOMB, softening=1e-3, alpha=200.0, affine=(0.0, 0.0, 0.0)):
        """Exact (mean, variance) of replay_cut's estimator per query, by enumeration."""
        q = _f32(queries, 3)
        mean = np.zeros(q.shape[0], np.float64)
        var = np.zeros(q.shape[0], np.float64)
        k = kernel(kind, softening, alpha, affine)
        self._lib.sbho_enumerate_cut(self._h, C.byref(k), _ptr(q), q.shape[0], C.c_float(beta_s), _ptr(mean), _ptr(var))
        return mean, var

    def enumerate(self, queries, kind=COULOMB, softening=1e-3, alpha=200.0, affine=(0.0, 0.0, 0.0),
                  sampling=SAMPLE_MASS, rr=RR_PAPER):
        """Exact (mean, variance) of the one-sample estimator per query, by enumeration."""
        q = _f32(queries, 3)
        mean = np.zeros(q.shape[0], np.float64)
        var = np.zeros(q.shape[0], np.float64)
        k = kernel(kind, softening, alpha, affine)
        o = _opts(sampling, rr, False)
        self._lib.sbho_enumerate(self._h, C.byref(k), _ptr(q), q.shape[0], C.byref(o), _ptr(mean), _ptr(var))
        return mean, var


MLP_NPARAM = 1313  # W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3


def mlp_forward(weights, feats) -> np.ndarray:
    """Scores of the learned proposal's 6-32-32-1 ReLU network (FP64) for feature rows [n, 6]."""
    lib = _load()
    w = np.ascontiguousarray(np.asarray(weights, np.float64))
    x = np.ascontiguousarray(np.asarray(feats, np.float64).reshape(-1, 6))
    out = np.zeros(x.shape[0], np.float64)
    lib.sbho_mlp_forward(_ptr(w), _ptr(x), x.shape[0], _ptr(out))
    return out


def mlp_loss_grad(weights, feats, targets, offsets):
    """Mean over decision sets of the cross-entropy between softmax(scores) and the normalised
    targets of each set (rows offsets[s]..offsets[s+1]-1), and its gradient (FP64)."""
    lib = _load()
    w = np.ascontiguousarray(np.asarray(weights, np.float64))
    x = np.ascontiguousarray(np.asarray(feats, np.float64).reshape(-1, 6))
    t = np.ascontiguousarray(np.asarray(targets, np.float64))
    off = np.ascontiguousarray(np.asarray(offsets, np.int64))
    g = np.zeros(MLP_NPARAM, np.float64)
    loss = lib.sbho_mlp_loss_grad(_ptr(w), _ptr(x), _ptr(t), _ptr(off), off.shape[0] - 1, _ptr(g))
    return float(loss), g


def max_threads() -> int:
    return int(_load().sbho_max_threads())


def set_threads(n: int) -> None:
    _load().sbho_set_threads(int(n))
