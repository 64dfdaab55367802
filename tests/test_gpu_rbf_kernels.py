"""The radial kernels of mf_rbf other than the Gaussian (Eq. rbfcoeff and
the tail-order rule after it) on the GPU against the FP64 oracle: the FP64
start-up (Cholesky for IMQ; the null-space method for the conditionally
definite PHS3 and MQ), the FP32 and tcgen05 evaluation, the columns-only
stage, a batch mixing kernels, and the argument checks."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu

# (kernel, overrides): eps twice the Gaussian's for MQ / IMQ (less cancellation
# in the interpolant's sum); eps = 1 for PHS3 (it only scales the kernel)
CASES = [
    ("phs3", "C0", {"kernel": "phs3", "eps": 1.0}),
    ("mq", "C0", {"kernel": "mq", "eps": 3.0}),
    ("mq0", "C0", {"kernel": "mq", "eps": 3.0, "tail_degree": 0}),
    ("imq", "C0", {"kernel": "imq", "eps": 3.0}),
    ("imq-", "C0", {"kernel": "imq", "eps": 3.0, "tail_degree": -1}),
    ("phs3", "C1", {"kernel": "phs3", "eps": 1.0}),
    ("mq", "C1", {"kernel": "mq", "eps": 4.0}),
    ("imq", "C1", {"kernel": "imq", "eps": 4.0}),
]


def _run(model, th, ex):
    import torch
    out = model.loglike(torch.from_numpy(th).cuda(), torch.from_numpy(ex).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _forms(kernel):
    # FP16 forms scale Phi by 2^14: only the kernels bounded by 1
    return ["fp32", "bf16_3term"] + (["fp16_3term"] if kernel in ("imq",) else [])


@pytest.mark.parametrize("tag,cfg,over", CASES, ids=[f"{c}-{t}" for t, c, _ in CASES])
def test_kernel_parity(tag, cfg, over):
    Q = 1931
    th, ex = _cases.queries(cfg, Q, seed=61, **over)
    ref = _cases.oracle_model(cfg, **over).loglike(th, ex)
    m = _cases.gpu_model(cfg, **over)
    assert np.all(np.isfinite(ref))
    for form in _forms(over["kernel"]):
        m.set_form(form)
        try:
            got = _run(m, th, ex)
            assert m.sync_status()[0] == 0
        finally:
            m.set_form("fp32")
        err = np.abs(got - ref)
        assert err.max() <= 0.01, (tag, cfg, form, err.max(), np.median(err))


@pytest.mark.parametrize("kernel", ["phs3", "mq"])
def test_fp16_forms_refuse_unbounded_kernels(kernel):
    import paper_2508_04172_gb300 as mf
    over = {"kernel": kernel, "eps": 1.0 if kernel == "phs3" else 3.0}
    m = _cases.gpu_model("C0", **over)
    for form in ("fp16", "fp16_wsplit", "fp16_3term"):
        with pytest.raises(mf.MFError) as e:
            m.set_form(form)
        assert e.value.code == mf.MF_E_NOTIMPL
    m.set_form("fp32")


@pytest.mark.parametrize("kernel,eps,tail", [("phs3", 1.0, 1), ("mq", 3.0, 1), ("mq", 3.0, 0), ("imq", 3.0, 1)])
def test_startup_weights_and_cond(kernel, eps, tail):
    """The sigma column (the same node data on both sides) against the
    oracle's LU solve of the saddle system, and the condition estimate of
    the matrix factored (Phi, or the projected one of the null-space method)."""
    import oracle
    over = {"kernel": kernel, "eps": eps, "tail_degree": tail}
    m = _cases.gpu_model("C0", **over)
    o = _cases.oracle_model("C0", **over)
    W, Wo = m.weights(), o.W
    s_col = o.F.shape[1] - 1
    assert np.abs(W[:, s_col] - Wo[:, s_col]).max() < 1e-8 * np.abs(Wo[:, s_col]).max()
    A = oracle.rbf_matrix(o.nodes, o.nodes, eps, kernel)
    if kernel in ("phs3", "mq"):
        N = A.shape[0]
        P = np.concatenate([np.ones((N, 1)), o.nodes], 1)[:, :oracle.tail_size(tail)]
        Qf, _ = np.linalg.qr(P, mode="complete")
        Z = Qf[:, P.shape[1]:]
        A = (-1.0 if kernel == "mq" else 1.0) * (Z.T @ A @ Z)
    c_ref = np.linalg.cond(A)
    assert 0.5 * c_ref <= m.query("cond") <= 1.01 * c_ref


@pytest.mark.parametrize("kernel,eps", [("phs3", 1.0), ("mq", 4.0)])
def test_columns_stage(kernel, eps):
    """mf_eval_columns (the Phi.W stage alone) against the oracle's
    interpolant fitted to the same node values (each side solves its own
    FP64 system); bound as for the Gaussian columns: the FP32 forward error
    of the length-(N+P) sum, gamma_(N+P) S with S = sum |a phi| + sum |b p|,
    plus the form's 16-bit splitting error."""
    import torch
    import oracle
    import paper_2508_04172_gb300 as mf
    over = {"kernel": kernel, "eps": eps}
    ev = _cases.event("C1", **over)
    s = ev.spec
    om = _cases.oracle_model("C1", **over)
    m = mf.Interpolant(om.nodes, om.F, eps, s.tail_degree, kernel=kernel)
    m.set_layout(s.n_det, s.n_modes, s.modes, s.rank)
    m.set_rotation(ev.metric, ev.centre)
    th, _ = _cases.queries("C1", 777, seed=62, **over)
    x = om.rotate(th.astype(np.float64))
    ref = om.rbf_eval(x)
    N = om.nodes.shape[0]
    P = om.W.shape[0] - N
    phi = np.abs(oracle.rbf_matrix(x, om.nodes, eps, kernel))
    tail = np.abs(np.concatenate([np.ones((len(x), 1)), x], axis=1)[:, :P])
    S = np.concatenate([phi, tail], axis=1) @ np.abs(om.W)
    split = {"fp32": 2.0 ** -21, "bf16_3term": 2.0 ** -15}
    try:
        for form in ("fp32", "bf16_3term"):
            m.set_form(form)
            got = m.eval_columns(torch.from_numpy(th).cuda()).cpu().numpy().astype(np.float64)
            d = np.abs(got - ref)
            bound = ((N + P) * 2.0 ** -24 + split[form]) * S + 1e-30
            worst = np.unravel_index(np.argmax(d / bound), d.shape)
            assert np.all(d <= bound), (kernel, form, worst, d[worst], bound[worst])
    finally:
        m.close()


def test_batch_mixing_kernels_equals_separate_calls():
    import torch
    import paper_2508_04172_gb300 as mf
    cases = [{"kernel": "gaussian"}, {"kernel": "phs3", "eps": 1.0}, {"kernel": "imq", "eps": 3.0}]
    ms, ths, exs = [], [], []
    for i, over in enumerate(cases):
        m = _cases.gpu_model("C0", **over)
        m.set_form("bf16_3term")
        th, ex = _cases.queries("C0", 500 + 211 * i, seed=63 + i, **over)
        ms.append(m)
        ths.append(torch.from_numpy(th).cuda())
        exs.append(torch.from_numpy(ex).cuda())
    try:
        sep = [m.loglike(t, e).cpu().numpy() for m, t, e in zip(ms, ths, exs)]
        b = mf.Batch(ms, [t.shape[0] for t in ths], autotune=False)
        got = [o.cpu().numpy() for o in b.loglike(ths, exs)]
        for a, c in zip(sep, got):
            assert np.array_equal(a, c)
        del b
    finally:
        for m in ms:
            m.set_form("fp32")


def test_tail_rule_and_kernel_id_checked():
    import paper_2508_04172_gb300 as mf
    rng = np.random.default_rng(64)
    nodes = rng.normal(size=(50, 4))
    F = rng.normal(size=(50, 2))
    for kernel, tail in (("phs3", 0), ("phs3", -1), ("mq", -1)):
        with pytest.raises(mf.MFError) as e:
            mf.Interpolant(nodes, F, 1.0, tail, kernel=kernel)
        assert e.value.code == mf.MF_E_INVAL
    with pytest.raises(mf.MFError) as e:
        mf.Interpolant(nodes, F, 1.0, 1, kernel=7)
    assert e.value.code == mf.MF_E_INVAL


def test_cpd_duplicate_nodes_are_refused():
    import paper_2508_04172_gb300 as mf
    rng = np.random.default_rng(65)
    nodes = rng.normal(size=(120, 4))
    nodes[90] = nodes[3]
    F = rng.normal(size=(120, 2))
    for kernel in ("phs3", "mq"):
        with pytest.raises(mf.MFError) as e:
            mf.Interpolant(nodes, F, 1.0, 1, kernel=kernel)
        assert e.value.code == mf.MF_E_ILLCOND
