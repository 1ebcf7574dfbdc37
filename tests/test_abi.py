"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hkv.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2603_17168_gb300 import SIGNATURES
from paper_2603_17168_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hkv_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = B.build_lib()
    try:
        return ctypes.CDLL(path)
    except OSError as e:  # no CUDA runtime on this machine at all
        pytest.skip(f"cannot load {path}: {e}")


def test_header_declares_the_boundary():
    names = declared_functions(os.path.join(ROOT, "include", "hkv.h"))
    for required in ("hkv_create", "hkv_destroy", "hkv_find", "hkv_contains",
                     "hkv_insert_or_assign", "hkv_assign", "hkv_erase", "hkv_size",
                     "hkv_export_batch", "hkv_set_step", "hkv_set_epoch", "hkv_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for header in sorted(os.listdir(os.path.join(ROOT, "include"))):
        for name in declared_functions(os.path.join(ROOT, "include", header)):
            assert hasattr(lib, name), f"{name} declared in include/{header} but not exported"


def test_binding_covers_the_header():
    names = set(declared_functions(os.path.join(ROOT, "include", "hkv.h")))
    assert names == set(SIGNATURES), names ^ set(SIGNATURES)


def test_last_error_is_callable_without_gpu(lib):
    lib.hkv_last_error.restype = ctypes.c_char_p
    assert lib.hkv_last_error() == b""


def test_invalid_arguments_fail_without_touching_the_gpu(lib):
    lib.hkv_create.restype = ctypes.c_int
    lib.hkv_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.hkv_create(None, None) == 1


def test_pipeline_refuses_bad_arguments_without_gpu(lib):
    lib.hkv_pipeline_create.restype = ctypes.c_int
    lib.hkv_pipeline_create.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                        ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.hkv_pipeline_create(0, 8, 3, ctypes.byref(h)) == 1      # no keys
    assert lib.hkv_pipeline_create(100, 8, 1, ctypes.byref(h)) == 1    # depth below 2
    assert lib.hkv_pipeline_create(100, 8, 9, ctypes.byref(h)) == 1    # depth above 8
    lib.hkv_pipeline_sync.restype = ctypes.c_int
    lib.hkv_pipeline_sync.argtypes = [ctypes.c_void_p]
    assert lib.hkv_pipeline_sync(None) == 1


def test_random_access_measurement_refuses_bad_arguments_without_gpu(lib):
    f = lib.hkv_measure_random_access
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                  ctypes.c_void_p]
    out = ctypes.c_double()
    assert f(16, 0, 1 << 30, 1 << 20, 1, ctypes.byref(out)) == 1       # unit not 8/32/128
    assert f(128, 0, (1 << 30) + 8, 1 << 20, 1, ctypes.byref(out)) == 1  # not a multiple of 128
    assert f(128, 0, 1 << 30, 0, 1, ctypes.byref(out)) == 1            # no accesses
    assert f(128, 0, 1 << 30, 1 << 20, 1, None) == 1                   # no output
