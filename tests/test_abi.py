"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/cld.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^CLD_API[^;(]*?\b(cld_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1503_06394_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_entry_points()
    for required in ("cld_create_csr", "cld_set_interval", "cld_estimate", "cld_grad", "cld_workspace_size",
                     "cld_set_workspace", "cld_auto_interval", "cld_destroy", "cld_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1503_06394_gb300 import _binding

    assert sorted(n for n, _, _ in _binding.SIGNATURES) == sorted(declared_entry_points())


def test_host_argument_checks_without_gpu(lib):
    from paper_1503_06394_gb300 import _binding as B

    B.load()
    h = ctypes.c_void_p()
    assert B.load().cld_create_csr(None, 4, 4, 1, 1, 1, 0, 0, None) == B.CLD_ERR_INVALID
    assert B.load().cld_create_csr(ctypes.byref(h), -1, 4, 1, 1, 1, 0, 0, None) == B.CLD_ERR_INVALID
    assert "negative" in B.cld_last_error()
    assert B.load().cld_create_csr(ctypes.byref(h), 4, 4, None, 1, 1, 0, 0, None) == B.CLD_ERR_INVALID
    assert B.load().cld_create_csr(ctypes.byref(h), 4, 4, 8, 8, 8, 9, 0, None) == B.CLD_ERR_INVALID
    assert B.load().cld_create_csr(ctypes.byref(h), 2**31, 4, 8, 8, 8, 0, 0, None) == B.CLD_ERR_INVALID
    # arrays not aligned to their element size (int64, int32, FP32 / BF16)
    assert B.load().cld_create_csr(ctypes.byref(h), 4, 4, 12, 8, 8, 0, 0, None) == B.CLD_ERR_INVALID
    assert "aligned" in B.cld_last_error()
    assert B.load().cld_create_csr(ctypes.byref(h), 4, 4, 8, 6, 8, 0, 0, None) == B.CLD_ERR_INVALID
    assert B.load().cld_create_csr(ctypes.byref(h), 4, 4, 8, 8, 6, 0, 0, None) == B.CLD_ERR_INVALID
    assert B.load().cld_create_csr(ctypes.byref(h), 4, 4, 8, 8, 7, 1, 0, None) == B.CLD_ERR_INVALID
    assert B.load().cld_set_interval(None, 0.1, 1.0) == B.CLD_ERR_INVALID
    assert B.load().cld_estimate(None, 3, 3, 0, None, None, None) == B.CLD_ERR_INVALID
    assert B.load().cld_version().startswith(b"libcld")


def test_missing_library_fails_loudly(tmp_path):
    from paper_1503_06394_gb300 import _binding as B

    saved = B._lib
    B._lib = None
    try:
        with pytest.raises(ImportError):
            B.load(str(tmp_path / "nope.so"))
    finally:
        B._lib = saved
