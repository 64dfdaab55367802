"""Polynomial tail degrees other than 1 (Eq. rbfcoeff with tail_degree 0:
a constant, and -1: no tail) on the GPU against the FP64 oracle built with
the same degree, in the plain FP32 form and a tcgen05 3-term form.

The plain FP32 form meets the 0.01 bar for every degree.  The 3-term form's
error scales with the cancellation in the weights (sum_n |a_n phi_n| over
max |F|): without a tail the Gaussians must also carry the affine part of
the data, and on C1 that ratio rises from 2.0e2 (degree 1) to 2.2e3, so the
FP16 3-term form (relative error about 2^-22 per product) is held to 0.03
there (measured 0.012); with a tail it meets 0.01."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu


def _run(model, th, ex):
    import torch
    out = model.loglike(torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("form", ["fp32", "fp16_3term"])
@pytest.mark.parametrize("cfg", ["C0", "C1"])
@pytest.mark.parametrize("tail", [0, -1])
def test_tail_degree_parity(cfg, tail, form):
    th, ex = _cases.queries(cfg, 1100, seed=31, tail_degree=tail)
    ref = _cases.oracle_model(cfg, tail_degree=tail).loglike(th, ex)
    m = _cases.gpu_model(cfg, tail_degree=tail)
    m.set_form(form)
    try:
        got = _run(m, th, ex)
        assert m.sync_status()[0] == 0
    finally:
        m.set_form("fp32")
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    bound = 0.03 if (form != "fp32" and tail == -1 and cfg != "C0") else 0.01
    assert err.max() <= bound, (cfg, tail, form, err.max())


def test_tail_degree_changes_the_fit():
    """The three degrees are different interpolants (the tail enters the
    solve): their lnL differ by far more than the rounding bar off the nodes."""
    th, ex = _cases.queries("C0", 256, seed=32)
    a = _run(_cases.gpu_model("C0", tail_degree=1), th, ex)
    b = _run(_cases.gpu_model("C0", tail_degree=0), th, ex)
    c = _run(_cases.gpu_model("C0", tail_degree=-1), th, ex)
    assert np.abs(a - b).max() > 0.03 and np.abs(a - c).max() > 0.03
