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
    finally:
        m.set_option("tc_pair", 1)
        m.set_form("fp32")
    assert np.all(np.isfinite(b))
    assert np.array_equal(a, b)
    if cfg == "C1":
        ref = _cases.oracle_model(cfg).loglike(th, ex)
        assert np.abs(b.astype(np.float64) - ref).max() <= 0.01
