"""The surrogate form's fused lnL epilogue, checked on its own: the network's
de-standardised output columns (mf_eval_columns in MF_FORM_MLP) are handed
to the FP64 oracle's time interpolation, amplitudes and quadratic form
(oracle.loglike_columns, Eqs. SVD, projected_h_fd, logl_complete), and the
surrogate form's lnL must match that to 1e-3 -- far below the network's own
approximation error, so a slip in the epilogue cannot hide behind the
held-out gate.

The library handle is built from the oracle's node values and SVD basis, so
the columns mean the same thing on both sides.  The network is trained
briefly: its accuracy is not what is tested here."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _handle_from_oracle(name):
    import paper_2508_04172_gb300 as mf
    ev = _cases.event(name)
    s = ev.spec
    om = _cases.oracle_model(name)
    m = mf.Interpolant(om.nodes, om.F, s.eps, s.tail_degree)
    m.set_layout(s.n_det, s.n_modes, s.modes, s.rank)
    m.set_basis(om.B, s.t0, s.dt)
    m.set_detectors(ev.det, s.d_ref)
    m.set_rotation(ev.metric, ev.centre)
    return m, om


@pytest.mark.parametrize("name", ["C1", "C4"])
def test_surrogate_epilogue_matches_oracle_on_network_columns(name):
    import torch
    import oracle
    m, om = _handle_from_oracle(name)
    try:
        tth, _ = _cases.queries(name, 20000, seed=81)
        hth, hex_ = _cases.queries(name, 2048, seed=82)
        st = m.train_surrogate(_cuda(tth), _cuda(hth), _cuda(hex_), steps=1500, seed=3,
                               gate_max=1e9, gate_median=1e9, r_gate=0.9)
        assert st["surrogate_gate"] == 1.0
        th, ex = _cases.queries(name, 1500, seed=83)      # 11 full tiles + a ragged one
        m.set_form("mlp")
        cols = m.eval_columns(_cuda(th))
        lnl = m.loglike(_cuda(th), _cuda(ex))
        torch.cuda.synchronize()
        assert m.sync_status()[0] == 0
        assert m.query("fallback_rate") == 0.0
        F = cols.cpu().numpy().astype(np.float64)
        got = lnl.cpu().numpy().astype(np.float64)
    finally:
        m.close()
    assert F.shape == (1500, om.K) and np.all(np.isfinite(F))
    ref = oracle.loglike_columns(om, F, ex)
    err = np.abs(got - ref)
    assert err.max() <= 1e-3, (name, err.max(), np.median(err))
