"""sbh_morton_sort_noalloc, the allocation-free Morton ordering for callers that cannot allocate
device memory (real-time loops that cannot take an allocation's synchronisation, applications that
own every allocation). Called through the C ABI; its output must equal what sbh_build computes
(sbh_tree_export's `code` and `perm`) bit for bit, on two calls in a row that share the library's
static scratch array, and sizes beyond SBH_NOALLOC_MAX_POINTS must be rejected."""
import ctypes

import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu
MAX_POINTS = 65536


def _noalloc(sbh, pts_np):
    import torch
    lib = sbh.load_library()
    fn = lib.sbh_morton_sort_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    n = pts_np.shape[0]
    P = dev(pts_np)
    codes = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    held, torch_held = sbh.sbh_memory_in_use(), torch.cuda.memory_allocated()
    st = fn(ctypes.c_void_p(P.data_ptr()), n, ctypes.c_void_p(codes.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, sbh.sbh_last_error()
    torch.cuda.synchronize()
    # the call took no memory from the library's allocator nor from torch's
    assert sbh.sbh_memory_in_use() == held and torch.cuda.memory_allocated() == torch_held
    return codes.cpu().numpy().view(np.uint64), perm.cpu().numpy()


def _reference(sbh, pts_np):
    w = np.ones(pts_np.shape[0], np.float32)
    t = sbh.sbh_build(dev(pts_np), dev(w))
    e = sbh.sbh_tree_export(t, 0)
    return e["code"], e["perm"]


def test_noalloc_sort_matches_build_on_consecutive_calls(sbh):
    rng = np.random.default_rng(2025)
    a = rng.random((MAX_POINTS, 3)).astype(np.float32)                       # the largest accepted size
    base = rng.normal(size=(900, 3)).astype(np.float32)
    b = base[rng.integers(0, 900, 3001)] + np.float32(1e-4) * rng.normal(size=(3001, 3)).astype(np.float32)
    b[::7] = b[3]                                                           # ties: order must stay stable
    for pts in (a, b, a):  # consecutive calls share the scratch array
        codes, perm = _noalloc(sbh, pts)
        rc, rp = _reference(sbh, pts)
        np.testing.assert_array_equal(codes, rc)
        np.testing.assert_array_equal(perm, rp)


def test_noalloc_sort_rejects_sizes_beyond_its_maximum(sbh):
    import torch
    lib = sbh.load_library()
    fn = lib.sbh_morton_sort_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    n = MAX_POINTS + 1
    P = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    codes = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    st = fn(ctypes.c_void_p(P.data_ptr()), n, ctypes.c_void_p(codes.data_ptr()), ctypes.c_void_p(perm.data_ptr()), None)
    assert st == 1 and "SBH_NOALLOC_MAX_POINTS" in sbh.sbh_last_error()
