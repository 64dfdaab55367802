"""Learned surrogate of the long-signal workload (one detector, four modes,
N = 8000 nodes, rank 80, M = 2048): the network trained on the GPU on 10^5
points labelled by the FP64 RBF interpolant, judged against the plain FP32
RBF path on 10^4 held-out queries, then checked against the FP64 oracle;
queries outside the training radius go to the RBF path unchanged, a failed
gate hands every query to the RBF path, and the network is much faster
than the method without it."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu

N_TRAIN, N_HELD = 100000, 10000


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def c4():
    m = _cases.gpu_model("C4")
    th, _ = _cases.queries("C4", N_TRAIN, seed=41)
    hth, hex_ = _cases.queries("C4", N_HELD, seed=42)
    stats = m.train_surrogate(_cuda(th), _cuda(hth), _cuda(hex_), seed=1)
    yield m, stats
    m.set_form("fp32")


def _run(m, th, ex):
    import torch
    out = m.loglike(_cuda(th), _cuda(ex))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def test_heldout_gate_passes(c4):
    m, st = c4
    assert st["surrogate_gate"] == 1.0, st
    assert st["surrogate_heldout_max"] <= 0.1 and st["surrogate_heldout_median"] <= 0.01, st
    assert 0.85 < st["surrogate_r_gate"] <= 0.9 + 1e-6
    assert st["surrogate_train_ms"] > 0 and st["surrogate_label_ms"] > 0


def test_surrogate_lnl_vs_oracle(c4):
    m, _ = c4
    th, ex = _cases.queries("C4", 4096, seed=43)
    m.set_form("mlp")
    try:
        got = _run(m, th, ex)
        assert m.sync_status()[0] == 0
        assert m.query("fallback_rate") <= 1e-3
    finally:
        m.set_form("fp32")
    idx = np.arange(0, 4096, 8)
    ref = _cases.oracle_model("C4").loglike(th[idx], ex[idx])
    err = np.abs(got[idx] - ref)
    assert err.max() <= 0.1 and np.median(err) <= 0.01, (err.max(), np.median(err))


def test_queries_beyond_training_radius_use_rbf(c4):
    m, st = c4
    ev = _cases.event("C4")
    th, ex = _cases.queries("C4", 3000, seed=44)
    d = th.astype(np.float64) - ev.centre
    r = np.linalg.norm(d, axis=1, keepdims=True)
    far = np.zeros(len(th), bool)
    far[::3] = True                      # a third pushed out to |x| = 0.95
    d[far] *= 0.95 / r[far]
    th2 = (ev.centre + d).astype(np.float32)
    ref = _run(m, th2, ex)               # fp32 RBF form
    m.set_form("mlp")
    try:
        got = _run(m, th2, ex)
        rate = m.query("fallback_rate")
    finally:
        m.set_form("fp32")
    assert rate == pytest.approx(far.mean(), abs=2e-3)
    # the same FP32 RBF kernel; the surrogate form lays the columns out in
    # narrower passes, so only the grouping of the passes' partial sums differs
    assert np.abs(got[far] - ref[far]).max() <= 1e-5 * max(1.0, np.abs(ref[far]).max())
    assert np.abs(got[~far] - ref[~far]).max() <= 0.1


def test_failed_gate_serves_rbf():
    """An undertrained network fails the held-out gate: the MLP form then
    returns exactly the plain FP32 RBF values."""
    m = _cases.gpu_model("C0")
    th, _ = _cases.queries("C0", 2048, seed=45)
    hth, hex_ = _cases.queries("C0", 512, seed=46)
    st = m.train_surrogate(_cuda(th), _cuda(hth), _cuda(hex_), steps=5, batch=256, hidden=64,
                           n_hidden=2, seed=2)
    assert st["surrogate_gate"] == 0.0
    q, e = _cases.queries("C0", 1000, seed=47)
    ref = _run(m, q, e)
    m.set_form("mlp")
    try:
        got = _run(m, q, e)
        assert m.query("fallback_rate") == 1.0
    finally:
        m.set_form("fp32")
    assert np.array_equal(got, ref)


def test_surrogate_speedup_over_plain_rbf(c4):
    """What the trained network gains: the same lnL (within the gate) at a
    fraction of the plain FP32 RBF path's time."""
    import torch
    m, _ = c4
    Q = 1 << 18
    th, ex = _cases.queries("C4", Q, seed=48)
    t, e = _cuda(th), _cuda(ex)
    out = torch.empty(Q, device="cuda")

    def timed(form, reps):
        m.set_form(form)
        m.loglike(t, e, out=out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            m.loglike(t, e, out=out)
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    try:
        t_rbf = timed("fp32", 2)
        t_mlp = timed("mlp", 5)
    finally:
        m.set_form("fp32")
    assert t_rbf / t_mlp > 5.0, (t_rbf, t_mlp)


def test_surrogate_form_call_captures_into_a_cuda_graph(c4):
    """The surrogate form sizes its RBF fallback launch on the device, so a
    whole call (network, fallback for queries beyond the training radius,
    scatter) enqueues without waiting for the GPU and can be captured; the
    replayed graph gives bit-identical lnL to a direct call."""
    import torch
    m, st = c4
    ev = _cases.event("C4")
    th, ex = _cases.queries("C4", 5000, seed=45)
    d = th.astype(np.float64) - ev.centre
    r = np.linalg.norm(d, axis=1, keepdims=True)
    far = np.zeros(len(th), bool)
    far[::5] = True                      # a fifth beyond the training radius
    d[far] *= 0.95 / r[far]
    th = (ev.centre + d).astype(np.float32)
    t, e = _cuda(th), _cuda(ex)
    m.set_form("mlp")
    try:
        direct = m.loglike(t, e).clone()
        torch.cuda.synchronize()
        rate = m.query("fallback_rate")
        out = torch.full_like(direct, float("nan"))
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            m.loglike(t, e, out=out)         # warm-up on the capture-side stream
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        out.fill_(float("nan"))
        with torch.cuda.graph(g):
            m.loglike(t, e, out=out)
        torch.cuda.synchronize()
        assert torch.isnan(out).all()        # captured, not run
        for _ in range(2):
            out.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(out, direct)
        assert m.sync_status()[0] == 0
    finally:
        m.set_form("fp32")
    assert abs(rate - far.mean()) <= 3.0 / len(th)    # (a stray in-ball query may sit beyond r_gate)
