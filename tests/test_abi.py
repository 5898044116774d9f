"""The C-ABI library loads and exports every entry point include/lgf.h declares.

No compute call is made here (these tests run without a GPU)."""

import ctypes
import os
import re

import pytest

from paper_1206_0675_gb300 import lgf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lgf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lgf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(lgf.LIB_PATH):
        from paper_1206_0675_gb300 import build
        build.build()
    return lgf.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lgf_create", "lgf_destroy", "lgf_set_links", "lgf_get_links", "lgf_step", "lgf_measure",
                     "lgf_fix", "lgf_get_transform", "lgf_status_string", "lgf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"liblgf.so does not export {name}"


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in lgf.SIGNATURES}
    assert bound == set(declared_functions())


def test_status_strings_without_gpu(lib):
    assert lib.lgf_status_string(0) == b"ok"
    assert lib.lgf_status_string(6) == b"not converged"
    assert lib.lgf_last_error(None) == b"null handle"


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    bad = (ctypes.c_int32 * 4)(5, 8, 8, 8)      # 5 is not 2^a 3^b
    assert lib.lgf_create(bad, 0, 0, None, ctypes.byref(h)) == lgf.LGF_E_UNSUPPORTED
    big = (ctypes.c_int32 * 4)(8, 8, 8, 256)    # above 128
    assert lib.lgf_create(big, 0, 0, None, ctypes.byref(h)) == lgf.LGF_E_UNSUPPORTED
    ok = (ctypes.c_int32 * 4)(8, 8, 8, 8)
    assert lib.lgf_create(ok, 7, 0, None, ctypes.byref(h)) == lgf.LGF_E_ARG   # bad precision
    assert lib.lgf_create(ok, 0, 1 << 9, None, ctypes.byref(h)) == lgf.LGF_E_ARG  # unknown flag
    assert lib.lgf_create(None, 0, 0, None, ctypes.byref(h)) == lgf.LGF_E_ARG
    assert lib.lgf_destroy(None) == 0
