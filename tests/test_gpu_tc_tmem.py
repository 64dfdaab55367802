"""The second tcgen05 design (RBF tile in tensor memory, one CTA per column
pass) against the cluster design and the FP64 oracle.  Where both designs
lay the columns out in the same passes the per-query arithmetic is the same
sequence of MMAs and epilogue steps, so the results must be bitwise equal."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu


def _run(m, th, ex):
    import torch
    out = m.loglike(torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _both(m, th, ex, form):
    m.set_form(form)
    try:
        m.set_option("tc_design", 0)
        a = _run(m, th, ex)
        assert m.query("tc_design") == 0
        m.set_option("tc_design", 1)
        b = _run(m, th, ex)
        assert m.query("tc_design") == 1
        st = m.sync_status()
    finally:
        m.set_option("tc_design", -1)
        m.set_form("fp32")
    return a, b, st


@pytest.mark.parametrize("form", ["bf16_3term", "fp16_3term", "fp16_wsplit", "bf16"])
def test_c1_designs_bitwise_equal(form):
    m = _cases.gpu_model("C1")
    th, ex = _cases.queries("C1", 2000, seed=61)        # 15 full tiles + a ragged one
    a, b, st = _both(m, th, ex, form)
    assert st[0] == 0
    assert np.array_equal(a, b)


def test_c1_tmem_design_vs_oracle():
    m = _cases.gpu_model("C1")
    th, ex = _cases.queries("C1", 1000, seed=62)
    _, b, _ = _both(m, th, ex, "fp16_3term")
    ref = _cases.oracle_model("C1").loglike(th, ex)
    assert np.abs(b - ref).max() <= 0.01


def test_c4_tmem_design_more_passes():
    """K = 656 needs 4 passes of <= 192 columns (3 in the cluster design):
    the passes' partial sums regroup, the result stays within rounding."""
    m = _cases.gpu_model("C4")
    th, ex = _cases.queries("C4", 700, seed=63)
    a, b, st = _both(m, th, ex, "fp16_3term")
    assert st[0] == 0
    assert np.abs(a - b).max() <= 1e-3
    ref = _cases.oracle_model("C4").loglike(th[:200], ex[:200])
    assert np.abs(b[:200] - ref).max() <= 0.01


def test_single_pass_picks_tmem_design():
    m = _cases.gpu_model("C0")
    th, ex = _cases.queries("C0", 1000, seed=64)
    m.set_form("fp16_3term")
    try:
        assert m.query("tc_design") == 1            # automatic: one pass
        got = _run(m, th, ex)
        m.set_option("tc_design", 0)
        other = _run(m, th, ex)
    finally:
        m.set_option("tc_design", -1)
        m.set_form("fp32")
    assert np.array_equal(got, other)
    ref = _cases.oracle_model("C0").loglike(th, ex)
    assert np.abs(got - ref).max() <= 0.01


def test_tmem_design_flags_out_of_window():
    m = _cases.gpu_model("C1")
    th, ex = _cases.queries("C1", 500, seed=65)
    ex = ex.copy()
    ex[::7, 4] = 1.0                                   # t_c far outside the sampled window
    m.set_form("bf16_3term")
    m.set_option("tc_design", 1)
    try:
        got = _run(m, th, ex)
        rc, n_bad = m.sync_status()
    finally:
        m.set_option("tc_design", -1)
        m.set_form("fp32")
    assert n_bad == len(range(0, 500, 7))
    assert np.all(np.isnan(got[::7]))
    mask = np.ones(500, bool)
    mask[::7] = False
    assert np.all(np.isfinite(got[mask]))
