"""C-ABI library: it builds for sm_103a, loads, and exports every entry point
declared in include/mf.h.  No compute call is made here (no GPU on CPU runs)."""
import ctypes
import os
import re

import pytest

import paper_2508_04172_gb300 as mf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    return sorted(set(re.findall(r"MF_API[^;(]*?\b(mf_\w+)\s*\(", src, flags=re.S)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mf_build", "mf_loglike", "mf_free", "mf_set_layout", "mf_set_basis",
              "mf_set_detectors", "mf_set_rotation", "mf_set_form", "mf_svd_compress",
              "mf_sync_status", "mf_query"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    so = mf.build()
    assert os.path.exists(so)
    L = ctypes.CDLL(so)
    for name in _declared():
        assert hasattr(L, name), name


def test_status_strings_without_gpu():
    L = mf.lib()
    assert L.mf_error_string(0) == b"MF_OK"
    assert b"MF_E_RANGE" in L.mf_error_string(-5)
    assert L.mf_version().startswith(b"mf ")


def test_invalid_arguments_are_rejected_before_any_device_work():
    L = mf.lib()
    h = ctypes.c_void_p()
    # NULL inputs / bad sizes -> MF_E_INVAL, no device touched
    assert L.mf_build(None, None, 10, 10, 0, 1.0, 1, None, ctypes.byref(h)) == -1
    assert L.mf_loglike(None, None, None, 16, 5, None, None) == -1
    assert L.mf_set_form(None, 0) == -1
    assert L.mf_svd_compress(None, 4, 4, 2, None, None, None, None) == -1
