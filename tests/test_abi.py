"""The C-ABI library builds, loads and exports every entry point that
include/gpspca.h declares (no GPU needed: nothing is called)."""

import ctypes
import os
import re

import pytest

from paper_1312_6182_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gpspca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(gpspca_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gpspca_create", "gpspca_solve", "gpspca_submit", "gpspca_poll", "gpspca_destroy",
                     "gpspca_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(binding.EXPORTED) | {"gpspca_last_error"}


def test_binding_loads_and_sets_signatures(lib_path):
    lib = binding.load(lib_path)
    assert lib.gpspca_solve.restype is ctypes.c_int
    assert lib.gpspca_last_error() is not None


def test_struct_layouts_match_the_header():
    # gpspca_matrix: void*, enum, enum, int64 x3, float*  -> 48 bytes on LP64
    assert ctypes.sizeof(binding.Matrix) == 48
    assert binding.Matrix.p.offset == 16 and binding.Matrix.col_scale.offset == 40
    # gpspca_out: enum (+pad), 7 pointers -> 64 bytes
    assert ctypes.sizeof(binding.Out) == 64
    assert binding.Out.X.offset == 8


def test_null_arguments_are_rejected_without_a_gpu(lib_path):
    lib = binding.load(lib_path)
    assert lib.gpspca_create(None, 0, 0, None) == binding.EINVAL
    assert lib.gpspca_solve(None, None, 0, None, 1, None, 1e-6, 10, None, 0, None) == binding.EINVAL
    assert lib.gpspca_poll(None, 1, 0) == binding.EINVAL
    assert lib.gpspca_destroy(None) == binding.OK
    assert b"NULL" in lib.gpspca_last_error()
    nc, best, dflt = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    assert lib.gpspca_tune(None, None, 0, None, 1, None, 0, 3, ctypes.byref(nc), ctypes.byref(best),
                           ctypes.byref(dflt)) == binding.EINVAL
    assert lib.gpspca_tune_save(None, b"/nonexistent/x") == binding.EINVAL
    assert lib.gpspca_tune_load(None, b"/nonexistent/x") == binding.EINVAL
