"""Parity at the larger workloads: C2 (N=4000, rank 40, every precision form)
and C4 (N=8000, rank 80, M=2048, four modes, one detector) on sampled
queries, each checked element by element against the FP64 oracle."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu

# per-form bounds on max |dlnL|: the forms the benchmark may choose (plain
# FP32 and both 3-term forms) must meet the 0.01 bar; the others are run and
# bounded loosely.
BOUND = {"fp32": 0.01, "fp16_3term": 0.01, "bf16_3term": 0.01,
         "fp16_wsplit": 5.0, "fp16": 5.0, "bf16_wsplit": 50.0, "bf16": 50.0}


def _run(model, th, ex):
    import torch
    out = model.loglike(torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def c2():
    th, ex = _cases.queries("C2", 1500, seed=21)
    return _cases.gpu_model("C2"), th, ex, _cases.oracle_model("C2").loglike(th, ex)


@pytest.mark.parametrize("form", list(BOUND))
def test_c2_form_parity(c2, form):
    m, th, ex, ref = c2
    m.set_form(form)
    try:
        got = _run(m, th, ex)
        assert m.sync_status()[0] == 0
    finally:
        m.set_form("fp32")
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    assert err.max() <= BOUND[form], (form, err.max(), np.quantile(err, 0.99))


@pytest.mark.parametrize("form", ["fp32", "fp16_3term"])
def test_c4_rbf_parity(form):
    th, ex = _cases.queries("C4", 700, seed=41)
    ref = _cases.oracle_model("C4").loglike(th, ex)
    m = _cases.gpu_model("C4")
    m.set_form(form)
    try:
        got = _run(m, th, ex)
        assert m.sync_status()[0] == 0
    finally:
        m.set_form("fp32")
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    assert err.max() <= 0.01, (form, err.max())
