"""The C ABI library builds for sm_103a, loads, and exports every function include/sbh.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sbh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sbh_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    from paper_2506_02219_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 9
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    lib.sbh_version.restype = ctypes.c_int32
    assert lib.sbh_version() == 1


def test_library_targets_sm_103a():
    from paper_2506_02219_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
