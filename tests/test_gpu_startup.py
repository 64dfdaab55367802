"""The FP64 start-up solve on the GPU (Eq. rbfcoeff with the side condition
P^T a = 0), by the library's own blocked Cholesky factorisation and
triangular solves: the weights reproduce the node values (the defining
property of an interpolant) on every column, satisfy the side condition,
agree with the oracle's dense LU solve of the saddle system, and a
numerically singular Gaussian matrix is refused with MF_E_ILLCOND."""
import numpy as np
import pytest

from tests import _cases

pytestmark = pytest.mark.gpu


def _phi(x, y, eps):
    return np.exp(-(eps ** 2) * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1))


@pytest.mark.parametrize("cfg,tail", [("C0", 1), ("C1", 1), ("C1", 0), ("C1", -1)])
def test_gpu_weights_reproduce_node_values(cfg, tail):
    import paper_2508_04172_gb300 as mf
    om = _cases.oracle_model(cfg, tail_degree=tail)
    s = _cases.event(cfg, tail_degree=tail).spec
    m = mf.Interpolant(om.nodes, om.F, s.eps, tail)
    try:
        W = m.weights()
    finally:
        m.close()
    N = om.nodes.shape[0]
    P = W.shape[0] - N
    assert P == {1: 5, 0: 1, -1: 0}[tail]
    tailm = np.concatenate([np.ones((N, 1)), om.nodes], axis=1)[:, :P]
    fit = _phi(om.nodes, om.nodes, s.eps) @ W[:N] + tailm @ W[N:]
    scale = np.abs(om.F).max()
    assert np.abs(fit - om.F).max() <= 1e-10 * scale, np.abs(fit - om.F).max() / scale
    if P:
        side = tailm.T @ W[:N]                     # P^T a = 0 for every column
        assert np.abs(side).max() <= 1e-10 * np.abs(W[:N]).sum(axis=0).max()
    # the oracle solves the same saddle system by dense LU with pivoting: the
    # two FP64 solutions agree to the conditioning of Phi
    cond = np.linalg.cond(_phi(om.nodes, om.nodes, s.eps))
    d = np.abs(W - om.W).max() / np.abs(om.W).max()
    assert d <= max(1e-12, 1e-14 * cond), (d, cond)


def test_gpu_condition_estimate_c1():
    m = _cases.gpu_model("C1")
    om = _cases.oracle_model("C1")
    s = _cases.event("C1").spec
    c_ref = np.linalg.cond(_phi(om.nodes, om.nodes, s.eps))
    assert 0.5 * c_ref <= m.query("cond") <= 1.01 * c_ref


def test_numerically_singular_matrix_is_refused():
    """N = 8000 nodes in the unit 4-ball with the wide Gaussian eps = 1.5:
    Phi is singular to FP64 rounding, so a pivot of the factorisation is not
    positive beyond rounding."""
    import paper_2508_04172_gb300 as mf
    from workload.standin import ball
    nodes = ball(np.random.default_rng(7), 8000)
    F = np.random.default_rng(8).standard_normal((8000, 3))
    with pytest.raises(mf.MFError) as e:
        mf.Interpolant(nodes, F, 1.5, 1)
    assert e.value.code == mf.MF_E_ILLCOND


def test_duplicate_nodes_are_refused():
    import paper_2508_04172_gb300 as mf
    from workload.standin import ball
    nodes = ball(np.random.default_rng(9), 300)
    nodes[200] = nodes[17]
    F = np.random.default_rng(10).standard_normal((300, 2))
    with pytest.raises(mf.MFError) as e:
        mf.Interpolant(nodes, F, 2.0, 1)
    assert e.value.code == mf.MF_E_ILLCOND
