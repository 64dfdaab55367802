"""Pins of the oracle's radial kernels (Eq. rbfcoeff and the tail rule after
it) against facts the mathematics fixes, not against retyped formulas:

* PHS3 with an affine tail, on nodes along one axis, is the natural cubic
  spline through the data (scipy's CubicSpline, bc 'natural');
* Gaussian, MQ and IMQ interpolants tend to the polynomial interpolant of the
  nodes as eps -> 0 (flat limit), with an error of order eps^2;
* signatures: Gaussian and IMQ matrices are positive definite, the MQ matrix
  has exactly one positive eigenvalue (Micchelli), the PHS3 matrix is
  indefinite but positive definite on the null space of the affine tail;
* polynomial reproduction: with a tail, the tail's polynomials are
  reproduced exactly (a = 0);
* a tail below the kernel's conditionally-positive-definite order is refused.
Evaluation goes through the C loops of mforacle.c (oracle.rbf_evaluate)."""
import numpy as np
import pytest

import oracle


def _axis_points(x):
    X = np.zeros((len(x), 4))
    X[:, 0] = x
    return X


def test_phs3_on_a_line_is_the_natural_cubic_spline():
    from scipy.interpolate import CubicSpline
    rng = np.random.default_rng(1)
    x = np.sort(rng.uniform(-2.0, 3.0, 14))
    f = np.sin(1.3 * x) + 0.2 * x ** 2
    xq = np.linspace(x[0], x[-1], 301)
    ref = CubicSpline(x, f, bc_type="natural")(xq)
    outs = []
    for eps in (0.8, 2.5):   # eps only scales the kernel: the same interpolant
        # fitted in one dimension (tail 1, x), evaluated by the 4-D loops on
        # the nodes' line (tail 1, x_1, 0, 0, 0)
        W1 = oracle.rbf_fit(x[:, None], f[:, None], eps, tail_degree=1, kernel="phs3")
        W = np.concatenate([W1, np.zeros((3, 1))])
        got = oracle.rbf_evaluate(_axis_points(x), W, eps, 1, _axis_points(xq), "phs3")[:, 0]
        assert np.abs(got - ref).max() < 1e-10 * np.abs(f).max()
        outs.append(got)
    assert np.abs(outs[0] - outs[1]).max() < 1e-10 * np.abs(f).max()


@pytest.mark.parametrize("kernel", ["gaussian", "mq", "imq"])
def test_flat_limit_is_the_polynomial_interpolant(kernel):
    x = np.array([-1.0, -0.45, 0.1, 0.6, 1.0])
    f = 1.0 + x - 0.5 * x ** 2 + 0.3 * x ** 3 + 0.7 * x ** 4
    xq = np.linspace(-1.0, 1.0, 41)
    poly = np.polyval(np.polyfit(x, f, len(x) - 1), xq)
    dev = []
    for eps in (0.2, 0.1):
        W = oracle.rbf_fit(_axis_points(x), f[:, None], eps, tail_degree=0, kernel=kernel)
        s = oracle.rbf_evaluate(_axis_points(x), W, eps, 0, _axis_points(xq), kernel)[:, 0]
        dev.append(np.abs(s - poly).max())
    assert dev[1] < 0.05 * np.abs(f).max()
    assert 3.0 < dev[0] / dev[1] < 5.0, dev   # O(eps^2)


def test_kernel_matrix_signatures():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(60, 4))
    for kernel in ("gaussian", "imq"):
        w = np.linalg.eigvalsh(oracle.rbf_matrix(X, X, 0.9, kernel))
        assert w.min() > 0, kernel
    w = np.linalg.eigvalsh(oracle.rbf_matrix(X, X, 0.9, "mq"))
    assert (w > 0).sum() == 1 and (w < 0).sum() == 59
    A = oracle.rbf_matrix(X, X, 0.9, "phs3")
    w = np.linalg.eigvalsh(A)
    assert w.min() < 0 < w.max()
    P = np.concatenate([np.ones((60, 1)), X], axis=1)
    Q, _ = np.linalg.qr(P, mode="complete")
    Z = Q[:, 5:]
    assert np.linalg.eigvalsh(Z.T @ A @ Z).min() > 0


@pytest.mark.parametrize("kernel,tail", [("phs3", 1), ("mq", 0), ("mq", 1), ("gaussian", 1), ("imq", 0)])
def test_tail_polynomials_reproduced(kernel, tail):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(40, 4))
    g = np.array([0.4, -1.1, 0.25, 2.0])
    f = 1.7 + (X @ g if tail == 1 else np.zeros(40))
    W = oracle.rbf_fit(X, f[:, None], 0.7, tail_degree=tail, kernel=kernel)
    assert np.abs(W[:40]).max() < 1e-9
    Xq = rng.normal(size=(25, 4))
    got = oracle.rbf_evaluate(X, W, 0.7, tail, Xq, kernel)[:, 0]
    assert np.abs(got - (1.7 + (Xq @ g if tail == 1 else 0.0))).max() < 1e-9


@pytest.mark.parametrize("kernel", oracle.RBF_KERNELS)
def test_nodes_reproduced(kernel):
    rng = np.random.default_rng(4)
    X = rng.normal(size=(50, 4))
    F = rng.normal(size=(50, 3))
    tail = max(1, oracle.min_tail_degree(kernel))
    W = oracle.rbf_fit(X, F, 0.8, tail_degree=tail, kernel=kernel)
    got = oracle.rbf_evaluate(X, W, 0.8, tail, X, kernel)
    assert np.abs(got - F).max() < 1e-8 * np.abs(F).max()
    assert np.abs(np.concatenate([np.ones((50, 1)), X], 1).T @ W[:50]).max() < 1e-8 * np.abs(W).max()


def test_tail_below_the_order_is_refused():
    X = np.random.default_rng(5).normal(size=(20, 4))
    F = np.ones((20, 1))
    assert oracle.min_tail_degree("phs3") == 1 and oracle.min_tail_degree("mq") == 0
    assert oracle.min_tail_degree("gaussian") == -1 and oracle.min_tail_degree("imq") == -1
    with pytest.raises(ValueError):
        oracle.rbf_fit(X, F, 1.0, tail_degree=0, kernel="phs3")
    with pytest.raises(ValueError):
        oracle.rbf_fit(X, F, 1.0, tail_degree=-1, kernel="mq")
