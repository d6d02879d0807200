"""The C ABI library loads and exports every entry point include/lrnr.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for fn in sorted(os.listdir(HEADER_DIR)):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(HEADER_DIR, fn)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^(?:const\s+)?(?:lrnr_status|void|char|int)\s*\*?\s*(\w+)\s*\(", src, re.M):
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2410_04001_gb300 import build as b
    b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_entry_points():
    names = set(declared_functions())
    for n in ("lrnr_build", "fastlrnr_select_rows", "lrnr_residual", "lrnr_residual_grad",
              "spinprop_step", "lrnr_last_device_status", "lrnr_status_string", "lrnr_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2410_04001_gb300 import binding
    assert set(declared_functions()) <= set(binding.EXPORTS)


def test_status_strings_without_a_gpu(lib):
    lib.lrnr_status_string.restype = ctypes.c_char_p
    assert lib.lrnr_status_string(0) == b"ok"
    assert b"invalid" in lib.lrnr_status_string(1)


def test_build_rejects_bad_arguments_without_touching_the_gpu(lib):
    out = ctypes.c_void_p()
    # L = 0 and null pointers are refused before any CUDA call
    assert lib.lrnr_build(0, 8, None, None, None, None, ctypes.byref(out)) == 1
    assert lib.lrnr_build(2, 8, None, None, None, None, ctypes.byref(out)) == 1
    r = (ctypes.c_int * 3)(2, 40, 1)   # rank above 32
    assert lib.lrnr_build(2, 8, r, None, None, None, ctypes.byref(out)) == 1


def test_copy_pinned_checks_arguments_before_any_cuda_call(lib):
    """lrnr_copy_pinned: an empty copy succeeds and a null pointer with bytes > 0 is
    refused, both before the library asks CUDA about the pointers."""
    f = lib.lrnr_copy_pinned
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    buf = ctypes.create_string_buffer(64)
    assert f(None, None, 0, None) == 0
    assert f(ctypes.addressof(buf), ctypes.addressof(buf), 0, None) == 0
    assert f(None, ctypes.addressof(buf), 64, None) == 1
    assert f(ctypes.addressof(buf), None, 64, None) == 1
