"""The Phi.W stage alone (mf_eval_columns), column by column, against the
FP64 oracle's interpolant (Eq. rbfcoeff) on the same node values.

Both sides fit the same node values F (the oracle's packed SVD coefficients
and cross terms), so every interpolated column is comparable; the library
solves its own FP64 system on the GPU.  The bound is the forward error of a
dot product of length N+P evaluated in FP32, gamma_(N+P) * S with
S = sum_n |a_n phi_n| + sum_p |b_p p_p| (the absolute sum of the terms),
plus the error of the form's 16-bit splitting of Phi and W (about 2^-22 of
S for the FP16 3-term form, 2^-16 for BF16, below 2^-21 for the FP32 form's
rounding of W and exp2); the columns that carry most of the signal are
also held to a relative bound against their own scale."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu

SPLIT = {"fp32": 2.0 ** -21, "fp16_3term": 2.0 ** -20, "bf16_3term": 2.0 ** -15}
REL_BIG = {"fp32": 0.01, "fp16_3term": 0.01, "bf16_3term": 0.05}


@pytest.fixture(scope="module")
def c1_same_values():
    import paper_2508_04172_gb300 as mf
    ev = _cases.event("C1")
    s = ev.spec
    om = _cases.oracle_model("C1")
    m = mf.Interpolant(om.nodes, om.F, s.eps, s.tail_degree)
    m.set_layout(s.n_det, s.n_modes, s.modes, s.rank)
    m.set_rotation(ev.metric, ev.centre)
    th, _ = _cases.queries("C1", 1931, seed=61)            # 15 full tiles + a ragged one
    x = om.rotate(th.astype(np.float64))
    ref = om.rbf_eval(x)
    N = om.nodes.shape[0]
    P = om.W.shape[0] - N
    phi = np.exp(-(s.eps ** 2) * ((x[:, None, :] - om.nodes[None, :, :]) ** 2).sum(-1))
    tail = np.concatenate([np.ones((len(x), 1)), x], axis=1)[:, :P]
    S = np.concatenate([phi, tail], axis=1) @ np.abs(om.W)
    yield m, th, ref, S, N + P
    m.close()


@pytest.mark.parametrize("form", ["fp32", "fp16_3term", "bf16_3term"])
def test_columns_match_oracle_interpolant(c1_same_values, form):
    import torch
    m, th, ref, S, n_terms = c1_same_values
    m.set_form(form)
    try:
        got = m.eval_columns(torch.from_numpy(th).cuda())
        torch.cuda.synchronize()
        got = got.cpu().numpy().astype(np.float64)
    finally:
        m.set_form("fp32")
    assert got.shape == ref.shape and np.all(np.isfinite(got))
    d = np.abs(got - ref)
    bound = (n_terms * 2.0 ** -24 + SPLIT[form]) * S + 1e-30
    worst = np.unravel_index(np.argmax(d / bound), d.shape)
    assert np.all(d <= bound), (form, worst, d[worst], bound[worst])
    scale = np.abs(ref).max(axis=0)
    big = scale >= 1e-3 * scale.max()
    rel = d[:, big].max(axis=0) / scale[big]
    assert rel.max() <= REL_BIG[form], (form, rel.max())


def test_columns_of_every_pass_are_written(c1_same_values):
    """Each device pass writes its own columns: no user column is left at
    the fill value in any form."""
    import torch
    m, th, _, _, _ = c1_same_values
    for form in ("fp32", "fp16_3term"):
        m.set_form(form)
        try:
            out = torch.full((64, m.K), float("nan"), device="cuda")
            m.eval_columns(torch.from_numpy(th[:64]).cuda(), out=out)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all(), form
        finally:
            m.set_form("fp32")
