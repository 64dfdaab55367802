"""Parity at the full workload sizes, in the launch configurations bench.py
times: C2 (Q = 262144), C4 (Q = 10^6) and the 100-event batch (one
persistent launch under a CUDA graph).  The FP64 oracle checks sampled
outputs one by one; every output is checked for the properties that hold at
any size (finite, no out-of-window count)."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu


def _full(name, form, n_check, seed):
    import torch
    spec = _cases.event(name).spec
    th, ex = _cases.queries(name, spec.Q)              # the bench's batch
    m = _cases.gpu_model(name)
    m.set_form(form)
    try:
        out = m.loglike(torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        rc, n_bad = m.sync_status()
    finally:
        m.set_form("fp32")
    assert rc == 0 and n_bad == 0
    assert got.shape == (spec.Q,) and np.all(np.isfinite(got))
    idx = np.sort(np.random.default_rng(seed).choice(spec.Q, n_check, replace=False))
    ref = _cases.oracle_model(name).loglike(th[idx], ex[idx])
    return np.abs(got[idx].astype(np.float64) - ref)


@pytest.mark.parametrize("form", ["bf16_3term", "fp16_3term"])
def test_c2_full_batch(form):
    err = _full("C2", form, 512, 71)
    assert err.max() <= 0.01, err.max()


def test_c4_full_batch():
    err = _full("C4", "fp16_3term", 256, 72)
    assert err.max() <= 0.01, err.max()


def test_c3_full_batch_one_launch():
    import torch
    import oracle
    import paper_2508_04172_gb300 as mf
    from workload import standin
    from workload.standin import c3_specs, make_event, make_queries
    specs = c3_specs()
    evs, models, th, ex = [], [], [], []
    for sp in specs:
        ev = make_event(sp)
        models.append(mf.Interpolant.from_overlaps(
            ev.nodes, standin.node_overlaps(ev), standin.standin_sigma(ev, ev.nodes), sp.rank,
            sp.eps, sp.modes, ev.det, sp.t0, sp.dt, sp.d_ref, ev.metric, ev.centre, sp.tail_degree,
            "fp16_3term"))
        a, b = make_queries(ev, sp.Q, seed=sp.seed + 17)     # the bench's batches
        evs.append(ev)
        th.append(a)
        ex.append(b)
    Qs = [sp.Q for sp in specs]
    b = mf.Batch(models, Qs, autotune=True)
    outs = b.loglike([torch.from_numpy(a).cuda() for a in th], [torch.from_numpy(c).cuda() for c in ex])
    torch.cuda.synchronize()
    rc, n_bad = b.sync_status()
    assert rc == 0 and n_bad == 0
    got = [o.cpu().numpy() for o in outs]
    for g, q in zip(got, Qs):
        assert g.shape == (q,) and np.all(np.isfinite(g))
    # sampled outputs of ten events spread over the draw (largest and smallest N, rank, Q among them)
    Ns = [sp.N for sp in specs]
    ranks = [sp.rank for sp in specs]
    picks = sorted({int(np.argmax(Ns)), int(np.argmin(Ns)), int(np.argmax(ranks)), int(np.argmin(ranks)),
                    int(np.argmax(Qs)), int(np.argmin(Qs)), 0, 33, 66, 99})
    for k in picks:
        idx = np.random.default_rng(k).choice(Qs[k], 64, replace=False)
        ref = oracle.Model.from_event(evs[k]).loglike(th[k][idx], ex[k][idx])
        err = np.abs(got[k][idx].astype(np.float64) - ref).max()
        assert err <= 0.01, (specs[k].name, err)
    b.close()
    for m in models:
        m.close()
