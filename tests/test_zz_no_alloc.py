"""mf_loglike_noalloc, the entry point for callers that cannot allocate device
memory during a call (fixed memory pools handed out at start-up, real-time
sampler loops that forbid allocation once they run).

It runs the same kernels as mf_loglike (plain FP32 form) in the same order,
so on consecutive calls that share its fixed scratch array it must return
bit-identical lnL; it must refuse batches whose partial sums would not fit.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu
TOL_FP32 = 0.01


def _noalloc(model, t, e, out):
    import torch
    import paper_2508_04172_gb300 as mf
    Q, E = e.shape
    st = torch.cuda.current_stream().cuda_stream
    return mf.lib().mf_loglike_noalloc(model._h, ctypes.c_void_p(t.data_ptr()),
                                       ctypes.c_void_p(e.data_ptr()), Q, E,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st))


def test_noalloc_matches_loglike_on_two_calls():
    import torch
    m = _cases.gpu_model("C1")
    m.set_form("fp32")
    assert m.query("n_pass") > 1          # the fixed scratch array is in use
    for seed, Q in ((3, 5000), (4, 4097)):
        th, ex = _cases.queries("C1", Q, seed=seed)
        t = torch.from_numpy(th).cuda()
        e = torch.from_numpy(ex).cuda()
        ref = m.loglike(t, e)
        out = torch.full((Q,), float("nan"), device="cuda")
        assert _noalloc(m, t, e, out) == 0
        torch.cuda.synchronize()
        a = out.cpu().numpy().astype(np.float64)
        b = ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= TOL_FP32
        assert np.array_equal(a, b)        # same kernels, same order: bit-identical


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    import paper_2508_04172_gb300 as mf
    m = _cases.gpu_model("C1")
    m.set_form("fp32")
    limit = 4194304
    Q = limit // int(m.query("n_pass")) + 1
    t = torch.zeros((Q, 4), device="cuda")
    e = torch.zeros((Q, 5), device="cuda")
    out = torch.zeros(Q, device="cuda")
    assert _noalloc(m, t, e, out) == mf.MF_E_INVAL
