"""The benchmark's measurement helpers (host only): log-log interpolation of time against error,
per-query error measures, error statistics, and the comment-blind kernel-source hash that decides
whether a committed ncu summary still describes the kernel."""
import os

import numpy as np

import bench


def test_interp_loglog_is_exact_on_power_laws_and_flags_extrapolation():
    xs = np.array([0.1, 0.01, 0.001])
    ys = 3.0 * xs ** -0.5  # time ~ error^-1/2
    for x in (0.05, 0.003):
        y, ex = bench.interp_loglog(x, xs, ys)
        assert abs(y - 3.0 * x ** -0.5) < 1e-9 * y and not ex
    y, ex = bench.interp_loglog(1e-4, xs, ys)  # beyond the sweep: extended along the last segment
    assert ex and abs(y - 3.0 * 1e-4 ** -0.5) < 1e-6 * y


def test_relative_error_forms():
    est, ref = np.array([1.1, 0.2]), np.array([1.0, 0.1])
    np.testing.assert_allclose(bench.rel_error("coulomb", est, ref), [0.1, 1.0])
    np.testing.assert_allclose(bench.rel_error("winding", est, ref), [0.1, 0.1])  # / max(|F|, 1)
    d = bench.rel_error("smoothdist", np.array([0.0011]), np.array([0.001]))
    np.testing.assert_allclose(d, [0.0001 / 0.002])  # / max(|d|, 2/1000)


def test_error_statistics():
    est = np.array([1.0, 2.0, np.inf, 4.0])
    ref = np.array([1.0, 1.0, 1.0, 1.0])
    s = bench.error_stats("coulomb", est, ref)
    assert s["non_finite"] == 1 and s["queries"] == 4
    assert s["rel"]["max"] == 3.0 and abs(s["rel"]["mean"] - 4.0 / 3.0) < 1e-12 and s["abs"]["median"] == 1.0
    t = bench.tail_errors(np.array([0.0, 1.0, 2.0, np.nan]))
    assert t["mean"] == 1.0 and 1.9 < t["p99"] <= 2.0


def test_source_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    a = tmp_path / "a.cu"
    a.write_text("int f() { return 1; } // one\n/* block\n comment */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_hash(["a.cu"])
    a.write_text("int f()  {\n  return 1;  }  // a different comment\n")
    assert bench.source_hash(["a.cu"]) == h0
    a.write_text("int f() { return 2; }\n")
    assert bench.source_hash(["a.cu"]) != h0


def test_committed_profile_matches_the_kernel_sources():
    # the estimator's ncu summary was taken on the kernel as it is now: the bench reports its traffic
    assert bench.profiled_bytes("winding") is not None
    assert bench.profiled_bytes("winding", "l2_bytes_per_query") is not None
    assert os.path.exists(os.path.join(bench.ROOT, "profiles", "launches_bench_winding.md"))


def test_every_hashed_profile_matches_the_kernel_sources():
    """Each committed ncu summary of a k_stoch_batched instance carries the hash of the kernel
    sources it was taken on; all must match the sources as they are now."""
    import glob
    want = bench.source_hash(bench.EVAL_SOURCES)
    paths = sorted(glob.glob(os.path.join(bench.ROOT, "profiles", "k_stoch_batched_*.md")))
    assert len(paths) >= 3
    for path in paths:
        first = open(path).readline().strip()
        assert first.startswith("<!-- source_hash="), path
        assert first == f"<!-- source_hash={want} -->", path


def test_fp32_peak_from_sm_count_and_clock():
    import bench
    # 152 SMs x 128 lanes x 2 flop x 2070 MHz
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9
    assert bench.peak_clock_mhz({"sm_max_mhz": 1965.0})[0] == 1965.0
    mhz, src = bench.peak_clock_mhz(None)
    assert mhz > 0 and src
