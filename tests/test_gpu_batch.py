"""Batched events: many interpolants with uneven node counts, SVD ranks and
batch sizes (drawn like the 100-event NSBH batch) evaluated by one persistent
tcgen05 launch replayed from a CUDA graph, with the launch shape chosen by the
library's autotuner.  Scheduling must not change any result: every event's
lnL equals the single-event launch of the same handle bit for bit, and the
FP64 oracle within the form's bound."""
import ctypes

import numpy as np
import pytest

from workload import standin
from workload.standin import c3_specs, make_event, make_queries

pytestmark = pytest.mark.gpu

IDX = [0, 1, 3, 4, 5, 7, 8]            # N 835..3635, rank 10..39
QS = [1000, 777, 1301, 129, 0, 2048, 513]   # ragged tails, one empty event
N_ORACLE = 150                          # sampled queries per event for the oracle


@pytest.fixture(scope="module")
def events():
    import torch
    import paper_2508_04172_gb300 as mf
    specs = c3_specs()
    out = []
    for i, Q in zip(IDX, QS):
        s = specs[i]
        ev = make_event(s)
        m = mf.Interpolant.from_overlaps(
            ev.nodes, standin.node_overlaps(ev), standin.standin_sigma(ev, ev.nodes), s.rank,
            s.eps, s.modes, ev.det, s.t0, s.dt, s.d_ref, ev.metric, ev.centre, s.tail_degree,
            "fp16_3term")
        th, ex = make_queries(ev, max(Q, 1), seed=s.seed + 99)
        th, ex = th[:Q], ex[:Q]
        out.append(dict(spec=s, ev=ev, model=m, th=th, ex=ex,
                        d_th=torch.from_numpy(np.ascontiguousarray(th)).cuda(),
                        d_ex=torch.from_numpy(np.ascontiguousarray(ex)).cuda()))
    return out


@pytest.fixture(scope="module")
def oracle_ref(events):
    import oracle
    ref = []
    for e in events:
        n = min(N_ORACLE, len(e["th"]))
        if n == 0:
            ref.append(np.empty(0))
            continue
        om = oracle.Model.from_event(e["ev"])
        ref.append(om.loglike(e["th"][:n], e["ex"][:n]))
    return ref


def _single(e):
    import torch
    if len(e["th"]) == 0:
        return np.empty(0)
    out = e["model"].loglike(e["d_th"], e["d_ex"])
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _host(outs):
    import torch
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("form", ["fp16_3term", "bf16"])
def test_batch_equals_single_launch(events, form):
    import paper_2508_04172_gb300 as mf
    for e in events:
        e["model"].set_form(form)
    try:
        b = mf.Batch([e["model"] for e in events], QS, autotune=True)
        got = _host(b.loglike([e["d_th"] for e in events], [e["d_ex"] for e in events]))
        assert b.sync_status()[0] == 0
        np_ = int(b.query("n_pass"))
        for e, g in zip(events, got):
            assert e["model"].query("n_pass") == np_
            ref = _single(e)
            assert g.shape == ref.shape
            assert np.all(np.isfinite(g))
            assert np.array_equal(g, ref), f"{e['spec'].name}: batch != single launch"
        b.close()
    finally:
        for e in events:
            e["model"].set_form("fp16_3term")


def test_batch_vs_oracle(events, oracle_ref):
    import paper_2508_04172_gb300 as mf
    b = mf.Batch([e["model"] for e in events], QS, autotune=True)
    got = _host(b.loglike([e["d_th"] for e in events], [e["d_ex"] for e in events]))
    assert b.sync_status()[0] == 0
    for e, g, ref in zip(events, got, oracle_ref):
        n = len(ref)
        if n == 0:
            assert g.size == 0
            continue
        err = np.abs(g[:n].astype(np.float64) - ref)
        assert err.max() <= 0.01, f"{e['spec'].name}: max |dlnL| {err.max():.3g}"
    b.close()


def test_graph_replay_and_recapture(events):
    import torch
    import paper_2508_04172_gb300 as mf
    b = mf.Batch([e["model"] for e in events], QS, autotune=False)
    th = [e["d_th"] for e in events]
    ex = [e["d_ex"] for e in events]
    outs = [torch.full((x.shape[0],), -1.0, device="cuda") for x in ex]
    b.loglike(th, ex, outs)
    first = _host(outs)
    for o in outs:
        o.fill_(-1.0)
    b.loglike(th, ex, outs)
    second = _host(outs)
    assert b.query("captures") == 1 and b.query("replays") == 1
    for a, c in zip(first, second):
        assert np.array_equal(a, c)
    # other sizes (a prefix of each event's queries): captured again
    cut = [x[: max(0, x.shape[0] - 37)] for x in th]
    cut_ex = [x[: max(0, x.shape[0] - 37)] for x in ex]
    o2 = b.loglike(cut, cut_ex)
    third = _host(o2)
    assert b.query("captures") == 2
    for a, c in zip(first, third):
        assert np.array_equal(a[: c.shape[0]], c)
    b.close()


def test_one_shot_matches_plan(events):
    import paper_2508_04172_gb300 as mf
    b = mf.Batch([e["model"] for e in events], QS, autotune=False)
    planned = _host(b.loglike([e["d_th"] for e in events], [e["d_ex"] for e in events]))
    b.close()
    once = _host(mf.loglike_batch([e["model"] for e in events], [e["d_th"] for e in events],
                                  [e["d_ex"] for e in events]))
    for a, c in zip(planned, once):
        assert np.array_equal(a, c)


def test_tuner_keeps_fastest_shape(events):
    import paper_2508_04172_gb300 as mf
    b = mf.Batch([e["model"] for e in events], QS, autotune=True)
    table = b.tuning()
    assert len(table) >= 1
    best = min(table, key=lambda t: t[2])
    assert (int(b.query("n_pass")), int(b.query("ring"))) == best[:2]
    for np_, ring, ms in table:
        assert 1 <= np_ <= 8 and 2 <= ring <= 4 and ms > 0
    b.close()


def test_changed_handle_invalidates_batch(events):
    import paper_2508_04172_gb300 as mf
    ms = [events[0]["model"], events[1]["model"]]
    b = mf.Batch(ms, QS[:2], autotune=False)
    ms[1].set_form("bf16_3term")
    try:
        with pytest.raises(mf.MFError) as ei:
            b.loglike([events[0]["d_th"], events[1]["d_th"]], [events[0]["d_ex"], events[1]["d_ex"]])
        assert ei.value.code == mf.MF_E_STATE
        # mixed forms cannot share one launch
        with pytest.raises(mf.MFError) as ei:
            mf.Batch(ms, QS[:2], autotune=False)
        assert ei.value.code == mf.MF_E_INVAL
    finally:
        ms[1].set_form("fp16_3term")
        b.close()


def test_batch_rejects_fp32_and_bad_args(events):
    import paper_2508_04172_gb300 as mf
    m = events[0]["model"]
    m.set_form("fp32")
    try:
        with pytest.raises(mf.MFError) as ei:
            mf.Batch([m], [100], autotune=False)
        assert ei.value.code == mf.MF_E_STATE
    finally:
        m.set_form("fp16_3term")
    L = mf.lib()
    out = ctypes.c_void_p()
    assert L.mf_batch_create(None, 1, None, 0, None, ctypes.byref(out)) == mf.MF_E_INVAL
    hs = (ctypes.c_void_p * 1)(m._h.value)
    neg = (ctypes.c_int * 1)(-5)
    assert L.mf_batch_create(hs, 1, neg, 0, None, ctypes.byref(out)) == mf.MF_E_INVAL
    assert L.mf_batch_create(hs, 0, neg, 0, None, ctypes.byref(out)) == mf.MF_E_INVAL


def test_misaligned_intrinsic_rejected(events):
    """Intrinsic rows are read as float4: a pointer off a 16-byte boundary
    is refused on the host before anything is launched."""
    import torch
    import paper_2508_04172_gb300 as mf
    e = events[0]
    m, th, ex = e["model"], e["d_th"], e["d_ex"]
    out = torch.empty(th.shape[0], device="cuda")
    L = mf.lib()
    P = ctypes.c_void_p
    rc = L.mf_loglike(m._h, P(th.data_ptr() + 4), P(ex.data_ptr()), th.shape[0] - 1, 5,
                      P(out.data_ptr()), None)
    assert rc == mf.MF_E_INVAL
    b = mf.Batch([m], [th.shape[0]], autotune=False)
    pi = (ctypes.c_void_p * 1)(th.data_ptr() + 8)
    pe = (ctypes.c_void_p * 1)(ex.data_ptr())
    po = (ctypes.c_void_p * 1)(out.data_ptr())
    q = (ctypes.c_int * 1)(th.shape[0] - 1)
    assert L.mf_batch_loglike(b._b, pi, pe, q, 5, po, None) == mf.MF_E_INVAL
    b.close()
