"""Device memory of the library: the caller's allocator and the memory cap.

- With PyTorch's caching allocator behind the library, a build and an evaluation give the same
  bits as with the library's own pool, the blocks show up in torch's accounting while the tree
  lives, and every byte is returned when it is freed.
- A memory cap below what a build needs makes sbh_build fail with SBH_ENOMEM and leak nothing;
  after the cap is lifted the same build succeeds.
"""
import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu


def _problem(n=50000, nq=4096, seed=3):
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    q = rng.random((nq, 3)).astype(np.float32)
    return pts, w, q


def test_torch_allocator_gives_the_same_results(sbh):
    import torch
    pts, w, q = _problem()
    P, M, Q = dev(pts), dev(w), dev(q)
    t0 = sbh.sbh_build(P, M)
    ref = sbh.sbh_eval(t0, Q, seed=5).cpu().numpy()
    bh_ref = sbh.sbh_eval_bh(t0, Q, theta=0.5).cpu().numpy()
    t0.free()
    torch.cuda.synchronize()
    base_lib = sbh.sbh_memory_in_use()
    before = torch.cuda.memory_allocated()
    sbh.use_torch_allocator()
    try:
        t = sbh.sbh_build(P, M)
        torch.cuda.synchronize()
        held = sbh.sbh_memory_in_use() - base_lib
        assert held > 0
        assert torch.cuda.memory_allocated() - before >= held
        out = sbh.sbh_eval(t, Q, seed=5).cpu().numpy()
        bh = sbh.sbh_eval_bh(t, Q, theta=0.5).cpu().numpy()
        assert np.array_equal(out, ref) and np.array_equal(bh, bh_ref)
        t.free()
        torch.cuda.synchronize()
        assert sbh.sbh_memory_in_use() == base_lib
        assert torch.cuda.memory_allocated() == before
    finally:
        sbh.sbh_set_allocator(None, None)


def test_memory_cap_makes_the_build_fail_cleanly(sbh):
    import torch
    pts, w, q = _problem()
    P, M, Q = dev(pts), dev(w), dev(q)
    torch.cuda.synchronize()
    base = sbh.sbh_memory_in_use()
    sbh.sbh_set_memory_limit(base + (1 << 20))  # 1 MB: a 50 k-point build needs several
    try:
        with pytest.raises(sbh.SBHError) as ei:
            sbh.sbh_build(P, M)
        assert ei.value.status == 2  # SBH_ENOMEM
        torch.cuda.synchronize()
        assert sbh.sbh_memory_in_use() == base
    finally:
        sbh.sbh_set_memory_limit(0)
    t = sbh.sbh_build(P, M)
    out = sbh.sbh_eval(t, Q, seed=5)
    assert bool(torch.isfinite(out).all())


def test_memory_cap_on_the_barnes_hut_tree(sbh):
    # the 8-ary tree is built on the first Barnes-Hut call: a cap there fails that call only
    import torch
    pts, w, q = _problem(seed=4)
    P, M, Q = dev(pts), dev(w), dev(q)
    t = sbh.sbh_build(P, M)
    torch.cuda.synchronize()
    held = sbh.sbh_memory_in_use()
    sbh.sbh_set_memory_limit(held + (1 << 16))
    try:
        with pytest.raises(sbh.SBHError) as ei:
            sbh.sbh_eval_bh(t, Q, theta=0.5)
        assert ei.value.status == 2
        torch.cuda.synchronize()
        assert sbh.sbh_memory_in_use() == held
    finally:
        sbh.sbh_set_memory_limit(0)
    out = sbh.sbh_eval_bh(t, Q, theta=0.5)
    ref = sbh.sbh_eval_bh(sbh.sbh_build(P, M), Q, theta=0.5)
    assert torch.equal(out, ref)
