"""The C ABI library builds, loads and exports every entry point that
include/bfsdf.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2602_19697_gb300 import bfsdf, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "bfsdf.h")).read()
    return re.findall(r"^(?:bf_status|void|int64_t|const char\*)\s+(bf_\w+)\(", hdr, re.M)


def test_library_exports_every_declared_entry_point():
    build.build()
    lib = bfsdf.load_library()
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(bfsdf.EXPORTED)


def test_null_arguments_are_rejected_without_touching_a_device():
    lib = bfsdf.load_library()
    assert lib.bf_create(0, None, None) == bfsdf.BF_EINVAL
    out = ctypes.c_void_p()
    assert lib.bf_build_band(None, None, 1, None, None, None, None, ctypes.byref(out)) == bfsdf.BF_EINVAL
    assert lib.bf_solve_mean(None, None, 1e-6, 10, 0, None, None, None) == bfsdf.BF_EINVAL
    assert lib.bf_band_info(None, None, None, None) == bfsdf.BF_EINVAL
    assert lib.bf_last_error(None) == b"null context"


def test_missing_library_fails_loudly(tmp_path):
    saved = bfsdf._lib
    bfsdf._lib = None
    try:
        try:
            bfsdf.load_library(str(tmp_path / "nope.so"))
        except RuntimeError as e:
            assert "no CPU fallback" in str(e)
        else:
            raise AssertionError("expected RuntimeError")
    finally:
        bfsdf._lib = saved
