"""GPU lnL (through the C ABI) against the FP64 oracle, element by element.

Bar: |dlnL| <= 0.01 for the plain FP32 form (the method's own accuracy
scale, Fig. logl_difference_plot medians 0.005-0.2)."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu
TOL_FP32 = 0.01


def _run(model, th, ex):
    import torch
    t = torch.from_numpy(th).cuda()
    e = torch.from_numpy(ex).cuda()
    out = model.loglike(t, e)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("Q", [1, 127, 1024, 1031])
def test_c0_parity_fp32(Q):
    th, ex = _cases.queries("C0", Q)
    ref = _cases.oracle_model("C0").loglike(th, ex)
    got = _run(_cases.gpu_model("C0"), th, ex)
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= TOL_FP32


def test_c1_parity_fp32_several_tiles_ragged():
    th, ex = _cases.queries("C1", 2000, seed=5)
    ref = _cases.oracle_model("C1").loglike(th, ex)
    got = _run(_cases.gpu_model("C1"), th, ex)
    err = np.abs(got - ref)
    assert err.max() <= TOL_FP32, (err.max(), np.median(err))


def test_c1_full_batch_sampled_parity_fp32():
    """Full C1 batch (Q = 65536, the benchmarked launch); 2048 sampled
    outputs checked against the oracle one by one."""
    th, ex = _cases.queries("C1", 65536)
    got = _run(_cases.gpu_model("C1"), th, ex)
    idx = np.random.default_rng(0).choice(65536, 2048, replace=False)
    ref = _cases.oracle_model("C1").loglike(th[idx], ex[idx])
    assert np.abs(got[idx] - ref).max() <= TOL_FP32
    assert np.all(np.isfinite(got))


def test_empty_batch_is_noop():
    import torch
    m = _cases.gpu_model("C0")
    out = torch.full((4,), 7.0, device="cuda")
    z = torch.empty((0, 4), device="cuda")
    e = torch.empty((0, 5), device="cuda")
    m.loglike(z, e, out=out[:0])
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)


def test_out_of_window_queries_are_nan_and_counted():
    m = _cases.gpu_model("C0")
    th, ex = _cases.queries("C0", 300)
    ex[10, 4] = 0.0155
    ex[200, 4] = -0.02
    ex[201, 4] = np.nan
    m.sync_status()
    got = _run(m, th, ex)
    rc, nbad = m.sync_status()
    assert np.isnan(got[10]) and np.isnan(got[200]) and np.isnan(got[201])
    assert np.isfinite(np.delete(got, [10, 200, 201])).all()
    assert rc == -5 and nbad == 3


def test_gpu_svd_matches_oracle_projection():
    import oracle
    import paper_2508_04172_gb300 as mf
    from workload import standin
    ev = _cases.event("C1")
    Z = standin.standin_z(ev, 2, 1, ev.nodes, ev.t_grid)
    C, B, sv = mf.svd_compress(Z, 20)
    Co, Bo, so = oracle.svd_compress(Z, 20)
    # the rank-l reconstruction is unique up to rounding of the noise subspace
    assert np.abs(C @ B - Co @ Bo).max() < 1e-7 * np.abs(Z).max()
    assert np.abs(sv[:8] - so[:8]).max() < 1e-6 * so[0]
    assert np.abs(B @ B.conj().T - np.eye(20)).max() < 1e-10


def test_gpu_rbf_weights_match_oracle_solve():
    m = _cases.gpu_model("C0")
    o = _cases.oracle_model("C0")
    W = m.weights()
    # columns differ only through the SVD basis choice; compare the tail-free
    # sigma column (same data on both sides) and node reproduction instead
    s_col = o.F.shape[1] - 1
    # cond estimate (power + inverse iteration) is a lower bound within 2x
    c_ref = np.linalg.cond(__import__("oracle").rbf_matrix(o.nodes, o.nodes, o.eps))
    assert 0.5 * c_ref <= m.query("cond") <= 1.01 * c_ref
    Wo = o.W
    assert np.abs(W[:, s_col] - Wo[:, s_col]).max() < 1e-6 * np.abs(Wo[:, s_col]).max()


def test_forms_report_passes():
    m = _cases.gpu_model("C1")
    assert m.query("n_pass") >= 3
    assert m.query("K") == 528


# --------------------------------------------------------------- tcgen05
TOL_CHOSEN = 0.01
# Expected accuracy of the other forms on C1 (probe of the arithmetic): the
# plain 16-bit and weight-split forms lose to the cancellation in the RBF
# weights (sum |a_n phi_n| / |F| ~ 1e5); they run, but are not chosen.
LOOSE = {"fp16_wsplit": 50.0, "bf16_wsplit": 500.0, "fp16": 50.0, "bf16": 500.0}


@pytest.mark.parametrize("form", ["fp16_3term", "bf16_3term"])
@pytest.mark.parametrize("cfg,Q", [("C0", 1031), ("C1", 1500), ("C1", 2000)])
def test_tc_3term_parity(cfg, Q, form):
    """The 3-term forms are the ones the benchmark may choose: both are held
    to the 0.01 bar on several tiles with a ragged last tile."""
    th, ex = _cases.queries(cfg, Q, seed=9 if Q != 2000 else 12)
    ref = _cases.oracle_model(cfg).loglike(th, ex)
    m = _cases.gpu_model(cfg)
    m.set_form(form)
    try:
        got = _run(m, th, ex)
        assert m.sync_status()[0] == 0
    finally:
        m.set_form("fp32")
    err = np.abs(got - ref)
    assert np.all(np.isfinite(got))
    assert err.max() <= TOL_CHOSEN, (form, err.max(), np.median(err))


@pytest.mark.parametrize("form", sorted(LOOSE))
def test_tc_other_forms_run_with_expected_accuracy(form):
    th, ex = _cases.queries("C1", 700, seed=10)
    ref = _cases.oracle_model("C1").loglike(th, ex)
    m = _cases.gpu_model("C1")
    m.set_form(form)
    try:
        got = _run(m, th, ex)
        assert m.sync_status()[0] == 0
    finally:
        m.set_form("fp32")
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= LOOSE[form]
