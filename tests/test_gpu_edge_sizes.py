"""Degenerate and extreme sizes of the online stage (Sec. II D), against the
FP64 oracle through the C ABI:

* an interpolant whose nodes, tail and padding all sit in the first node
  block (N = 12, one detector, one mode);
* fewer node blocks than column passes (N = 40 with the 3-detector,
  4-mode layout: 2 node blocks, 3 passes), so some CTAs of a cluster make no
  RBF tile at all, in every design and launch shape;
* the largest batch the entry points take (Q = 2^26, C1 layout, partial sums
  of 3 passes indexed past 2^31 bytes) and the first one they refuse.

The GPU interpolants are fitted by the library to the oracle's own node
values (the oracle's SVD needs no more nodes than samples)."""
import ctypes

import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu
TOL = 0.01
QMAX = 1 << 26


def _from_oracle(name, **over):
    import paper_2508_04172_gb300 as mf
    ev = _cases.event(name, **over)
    s = ev.spec
    om = _cases.oracle_model(name, **over)
    m = mf.Interpolant(om.nodes, om.F, s.eps, s.tail_degree)
    m.set_layout(s.n_det, s.n_modes, s.modes, s.rank)
    m.set_basis(om.B, s.t0, s.dt)
    m.set_detectors(ev.det, s.d_ref)
    m.set_rotation(ev.metric, ev.centre)
    return m, om


def _run(m, th, ex):
    import torch
    out = m.loglike(torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda())
    torch.cuda.synchronize()
    rc, n_bad = m.sync_status()
    assert rc == 0 and n_bad == 0
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("form,design", [("fp32", -1), ("bf16_3term", -1), ("fp16_3term", -1),
                                         ("bf16_3term", 0), ("fp16_3term", 0)])
def test_nodes_tail_and_padding_in_one_block(form, design):
    over = dict(N=12)
    m, om = _from_oracle("C0", **over)
    th, ex = _cases.queries("C0", 300, seed=81, **over)
    ref = om.loglike(th, ex)
    try:
        m.set_form(form)
        if form != "fp32":
            m.set_option("tc_design", design)
        got = _run(m, th, ex)
    finally:
        m.close()
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= TOL


@pytest.mark.parametrize("form,option,value", [
    ("fp32", None, None),
    ("bf16_3term", "tc_pair", 1), ("bf16_3term", "tc_pair", 0), ("bf16_3term", "tc_design", 1),
    ("fp16_3term", "tc_pair", 1), ("fp16_3term", "tc_pair", 0), ("fp16_3term", "tc_design", 1)])
def test_fewer_node_blocks_than_passes(form, option, value):
    over = dict(N=40, eps=2.0)
    m, om = _from_oracle("C1", **over)
    th, ex = _cases.queries("C1", 1000, seed=82, **over)
    ref = om.loglike(th, ex)
    try:
        m.set_form(form)
        if option is not None:
            m.set_option(option, value)
        got = _run(m, th, ex)
        if form != "fp32":
            assert m.query("n_pass") == 3
    finally:
        m.close()
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= TOL


@pytest.mark.parametrize("form", ["fp32", "bf16_3term"])
def test_largest_batch(form):
    import torch
    base = 1 << 20
    th, ex = _cases.queries("C1", base, seed=83)
    t = torch.from_numpy(th).cuda().repeat(QMAX // base, 1)
    e = torch.from_numpy(ex).cuda().repeat(QMAX // base, 1)
    assert t.shape[0] == QMAX
    m = _cases.gpu_model("C1")
    m.sync_status()                       # clear counts left by earlier calls on the shared model
    try:
        m.set_form(form)
        out = m.loglike(t, e)
        torch.cuda.synchronize()
        rc, n_bad = m.sync_status()
        if form != "fp32":
            assert m.query("n_pass") == 3
    finally:
        m.set_form("fp32")
    assert rc == 0 and n_bad == 0
    assert bool(torch.isfinite(out).all())
    rng = np.random.default_rng(84)
    idx = np.unique(np.concatenate([rng.choice(QMAX, 384, replace=False),
                                    np.arange(QMAX - 128, QMAX)]))
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    ref = _cases.oracle_model("C1").loglike(th[idx % base], ex[idx % base])
    assert np.abs(got - ref).max() <= TOL
    del t, e, out
    torch.cuda.empty_cache()


def test_batches_beyond_the_largest_are_refused():
    """Q = 2^26 + 1 is refused on the host before any pointer is used."""
    import torch
    import paper_2508_04172_gb300 as mf
    m = _cases.gpu_model("C1")
    t = torch.zeros((4, 4), device="cuda")
    e = torch.zeros((4, 5), device="cuda")
    out = torch.zeros(4, device="cuda")
    P = ctypes.c_void_p
    st = P(torch.cuda.current_stream().cuda_stream)
    L = mf.lib()
    q = QMAX + 1
    assert L.mf_loglike(m._h, P(t.data_ptr()), P(e.data_ptr()), q, 5, P(out.data_ptr()), st) == mf.MF_E_INVAL
    assert L.mf_eval_columns(m._h, P(t.data_ptr()), q, P(out.data_ptr()), st) == mf.MF_E_INVAL
    assert L.mf_loglike_noalloc(m._h, P(t.data_ptr()), P(e.data_ptr()), q, 5, P(out.data_ptr()),
                                st) == mf.MF_E_INVAL
    torch.cuda.synchronize()
    assert torch.all(out == 0)


def test_batch_member_with_fewer_node_blocks_than_passes():
    """One persistent launch over a 2-block interpolant (N = 40, 3 passes) and
    the full C1 interpolant, with batches of 1, 129 and 2000 queries: each
    event equals its own single launch bit for bit, and the oracle within the
    bound."""
    import torch
    import paper_2508_04172_gb300 as mf
    over = dict(N=40, eps=2.0)
    tiny, om_tiny = _from_oracle("C1", **over)
    big, om_big = _cases.gpu_model("C1"), _cases.oracle_model("C1")
    members = [(tiny, om_tiny, over, 1), (big, om_big, {}, 129), (tiny, om_tiny, over, 2000),
               (big, om_big, {}, 1)]
    hq = [_cases.queries("C1", q, seed=90 + i, **o) for i, (_, _, o, q) in enumerate(members)]
    dth = [torch.from_numpy(th).cuda() for th, _ in hq]
    dex = [torch.from_numpy(ex).cuda() for _, ex in hq]
    b = None
    try:
        for m in (tiny, big):
            m.set_form("bf16_3term")
        b = mf.Batch([m for m, _, _, _ in members], [q for _, _, _, q in members], autotune=False)
        outs = b.loglike(dth, dex)
        torch.cuda.synchronize()
        assert b.sync_status()[0] == 0
        assert int(b.query("n_pass")) == 3
        got = [o.cpu().numpy() for o in outs]
        single = []
        for (m, _, _, _), t, e in zip(members, dth, dex):
            single.append(m.loglike(t, e).cpu().numpy())
    finally:
        if b is not None:
            b.close()                     # before its members
        big.set_option("pass_count", 0)   # the batch fixed its members' pass count: back to automatic
        big.set_form("fp32")
        tiny.close()
    for (m, om, _, q), (th, ex), g, s in zip(members, hq, got, single):
        assert g.shape == (q,) and np.all(np.isfinite(g))
        assert np.array_equal(g, s)
        assert np.abs(g.astype(np.float64) - om.loglike(th, ex)).max() <= TOL


@pytest.mark.parametrize("cfg", ["C1", "C1S"])
@pytest.mark.parametrize("form", ["fp32", "bf16_3term"])
def test_extreme_extrinsics(cfg, form):
    """The ends of every extrinsic range: face-on and face-away (cos iota =
    +-1, one helicity only), psi = 0 and pi, phi_c = 0 and 2 pi, d_L at both
    ends of the prior, and with sky-dependent patterns a source at either
    celestial pole and alpha = 0 and 2 pi: the oracle within the bound."""
    th, ex = _cases.queries(cfg, 840, seed=95)
    ex = ex.copy()
    ex[0::4, 1], ex[1::4, 1] = 1.0, -1.0
    ex[0::3, 2], ex[1::3, 2] = 0.0, np.float32(np.pi)
    ex[0::5, 3], ex[1::5, 3] = 0.0, np.float32(2 * np.pi)
    ex[0::7, 0], ex[1::7, 0] = 100.0, 400.0
    if ex.shape[1] >= 7:
        ex[0::6, 6], ex[1::6, 6] = np.float32(np.pi / 2), np.float32(-np.pi / 2)
        ex[0::8, 5], ex[1::8, 5] = 0.0, np.float32(2 * np.pi)
    m = _cases.gpu_model(cfg)
    m.sync_status()
    try:
        m.set_form(form)
        got = _run(m, th, ex)
    finally:
        m.set_form("fp32")
    assert np.all(np.isfinite(got))
    assert np.abs(got - _cases.oracle_model(cfg).loglike(th, ex)).max() <= TOL
