"""The paired tcgen05 launch (two query tiles per cluster; each weight tile
multicast to both tiles' CTAs of a column pass) against the single launch:
per query the arithmetic and its order are the same, so the results must be
bitwise equal, ragged last pair included; and against the FP64 oracle."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu


def _run(m, th, ex):
    import torch
    out = m.loglike(torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("cfg,Q", [("C1", 2000), ("C1", 3 * 128 + 5), ("C4", 1931)])
@pytest.mark.parametrize("form", ["bf16_3term", "fp16_3term"])
def test_paired_launch_bitwise_equal_to_single(cfg, Q, form):
    m = _cases.gpu_model(cfg)
    th, ex = _cases.queries(cfg, Q, seed=71)
    m.set_form(form)
    try:
        m.set_option("tc_pair", 0)
        a = _run(m, th, ex)
        m.set_option("tc_pair", 1)
        b = _run(m, th, ex)
        assert m.sync_status()[0] == 0
        assert m.query("tc_paired") == 1   # 3 passes: clusters of 6 CTAs are paired
    finally:
        m.set_option("tc_pair", 1)
        m.set_form("fp32")
    assert np.all(np.isfinite(b))
    assert np.array_equal(a, b)
    if cfg == "C1":
        ref = _cases.oracle_model(cfg).loglike(th, ex)
        assert np.abs(b.astype(np.float64) - ref).max() <= 0.01


def test_pairing_skipped_when_clusters_of_eight_idle_sms():
    """4 passes would pair into clusters of 8 CTAs, which leave more SMs idle
    than clusters of 4 on this GPU: the launch stays single (same results)."""
    m = _cases.gpu_model("C2", N=1500, M=512)
    th, ex = _cases.queries("C2", 700, seed=72, N=1500, M=512)
    try:
        m.set_form("bf16_3term")
        assert m.query("n_pass") == 4
        _run(m, th, ex)
        assert m.query("tc_paired") == 0
    finally:
        m.set_form("fp32")


def test_chunked_cluster_launches_equal_one_launch():
    """A layout of 4 passes run as one cluster launch and as two launches of
    2 passes each (option tc_chunk) gives bitwise the same lnL: every pass
    partial is computed the same way, then summed in pass order."""
    import torch
    m = _cases.gpu_model("C2", N=1500, M=512)
    th, ex = _cases.queries("C2", 1931, seed=71, N=1500, M=512)
    d_th, d_ex = torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda()
    try:
        for form in ("bf16_3term", "fp16"):
            m.set_form(form)
            m.set_option("pass_count", 4)
            assert m.query("n_pass") == 4
            one = m.loglike(d_th, d_ex).cpu().numpy()
            m.set_option("tc_chunk", 2)
            two = m.loglike(d_th, d_ex).cpu().numpy()
            cols1 = m.eval_columns(d_th[:300]).cpu().numpy()
            m.set_option("tc_chunk", 0)
            cols0 = m.eval_columns(d_th[:300]).cpu().numpy()
            assert np.array_equal(one, two), form
            assert np.array_equal(cols0, cols1), form
    finally:
        m.set_option("tc_chunk", 0)
        m.set_option("pass_count", 0)
        m.set_form("fp32")
