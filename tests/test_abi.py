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


def test_batch_network_and_surrogate_entry_points_reject_bad_arguments():
    """The batched-events, network and surrogate entry points validate their
    arguments on the host before any device work."""
    L = mf.lib()
    P = ctypes.c_void_p
    out = P()
    q = (ctypes.c_int * 1)(16)
    # batched events: no handles, empty or oversized batches, NULL plan / output
    assert L.mf_batch_create(None, 1, q, 0, None, ctypes.byref(out)) == mf.MF_E_INVAL
    assert L.mf_batch_create(None, 0, q, 0, None, ctypes.byref(out)) == mf.MF_E_INVAL
    assert L.mf_batch_create(None, 129, q, 0, None, ctypes.byref(out)) == mf.MF_E_INVAL
    assert L.mf_batch_create(None, 1, q, 0, None, None) == mf.MF_E_INVAL
    assert L.mf_batch_loglike(None, None, None, q, 5, None, None) == mf.MF_E_INVAL
    assert L.mf_batch_set_option(None, b"graph", 0.0) == mf.MF_E_INVAL
    v = ctypes.c_double()
    assert L.mf_batch_query(None, b"n_pass", ctypes.byref(v)) == mf.MF_E_INVAL
    assert L.mf_batch_tuning(None, 0, None, None, None) == mf.MF_E_INVAL
    L.mf_batch_free(None)                          # no-op
    # network: every dimension limit of mf_mlp_create
    for dims in ((0, 256, 3, 656), (17, 256, 3, 656), (4, 8, 3, 656), (4, 100, 3, 656),
                 (4, 272, 3, 656), (4, 256, 0, 656), (4, 256, 8, 656), (4, 256, 3, 650),
                 (4, 256, 3, 0)):
        assert L.mf_mlp_create(*dims, 0, ctypes.byref(out)) == mf.MF_E_INVAL, dims
    assert L.mf_mlp_create(4, 256, 3, 656, 0, None) == mf.MF_E_INVAL
    assert L.mf_mlp_n_params(None) == -1
    assert L.mf_mlp_set_params(None, None) == mf.MF_E_INVAL
    assert L.mf_mlp_forward(None, None, 16, None, None) == mf.MF_E_INVAL
    assert L.mf_mlp_gradient(None, None, None, 16, None, None, None) == mf.MF_E_INVAL
    assert L.mf_mlp_query(None, b"loss", ctypes.byref(v)) == mf.MF_E_INVAL
    L.mf_mlp_free(None)
    # surrogate training: no handle / no data / no parameters
    sp = mf.SurrogateParams()
    assert L.mf_train_surrogate(None, None, 1000, None, None, 0, 5, ctypes.byref(sp), None) == mf.MF_E_INVAL
    # the no-allocation path and the column evaluation reject NULL handles too
    assert L.mf_loglike_noalloc(None, None, None, 16, 5, None, None) == mf.MF_E_INVAL
    assert L.mf_eval_columns(None, None, 16, None, None) == mf.MF_E_INVAL


def test_no_cpu_fallback_without_a_device():
    """With valid arguments but no CUDA device, the library fails with
    MF_E_CUDA instead of computing anything on the host, and the binding
    turns that into an exception."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    L = mf.lib()
    rng = np.random.default_rng(0)
    nodes = rng.uniform(-0.5, 0.5, (40, 4))
    vals = rng.standard_normal((40, 3))
    h = ctypes.c_void_p()
    rc = L.mf_build(nodes.ctypes.data, vals.ctypes.data, 40, 3, mf.RBF_KERNELS.index("gaussian"), 1.5, 1, None,
                    ctypes.byref(h))
    assert rc == mf.MF_E_CUDA and not h.value
    with pytest.raises(mf.MFError):
        mf.Interpolant(nodes, vals, 1.5, 1)


def test_binding_raises_when_the_library_is_missing(monkeypatch, tmp_path):
    """No silent fallback in the binding either: without libmf.so it raises."""
    monkeypatch.setattr(mf, "_lib", None)
    monkeypatch.setattr(mf, "_SO_PATH", str(tmp_path / "libmf.so"))
    with pytest.raises(RuntimeError, match="not built"):
        mf.lib()
