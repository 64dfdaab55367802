"""Pins of the FP64 surrogate-network reference against what fixes it
independently of its own code: central finite differences of the loss,
closed forms of SiLU and of Adam's first steps, structural zeros, and the
permutation symmetry of hidden units."""
import numpy as np
import pytest

from oracle import mlp


def _net(rng, n_in=4, hidden=7, n_hidden=3, n_out=5, scale=0.6):
    return [(rng.standard_normal((o, i)) * scale, rng.standard_normal(o) * 0.3)
            for o, i in mlp.shapes(n_in, hidden, n_hidden, n_out)]


def test_silu_closed_forms():
    assert mlp.silu(0.0) == 0.0
    assert mlp.silu_grad(0.0) == pytest.approx(0.5, abs=1e-15)
    z = np.array([-30.0, -2.0, 0.3, 2.0, 30.0])
    # SiLU(z) = z / (1 + e^-z): large z -> z, large -z -> 0
    assert mlp.silu(30.0) == pytest.approx(30.0, rel=1e-12)
    assert abs(mlp.silu(-30.0)) < 1e-11
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, rtol=1e-8, atol=1e-12)


def test_gradients_equal_finite_differences():
    rng = np.random.default_rng(0)
    params = _net(rng)
    x = rng.standard_normal((6, 4))
    t = rng.standard_normal((6, 5))
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t)
    flat = mlp.flatten(params)
    g_flat = mlp.flatten(grads)
    h = 1e-6
    for k in range(flat.size):
        p = flat.copy()
        p[k] += h
        lp = mlp.loss(mlp.forward(mlp.unflatten(p, 4, 7, 3, 5), x)[0], t)
        p[k] -= 2 * h
        lm = mlp.loss(mlp.forward(mlp.unflatten(p, 4, 7, 3, 5), x)[0], t)
        fd = (lp - lm) / (2 * h)
        assert abs(g_flat[k] - fd) <= 1e-6 * max(1e-3, abs(fd)), (k, g_flat[k], fd)


def test_output_bias_gradient_is_mean_residual():
    rng = np.random.default_rng(1)
    params = _net(rng)
    x = rng.standard_normal((9, 4))
    t = rng.standard_normal((9, 5))
    y, cache = mlp.forward(params, x)
    grads = mlp.backward(params, cache, y, t)
    # d/db_L of mean (y - t)^2 = 2 sum_b (y_b - t_b) / (B K)
    assert np.allclose(grads[-1][1], 2 * (y - t).sum(0) / (9 * 5), rtol=1e-13, atol=1e-15)


def test_zero_output_layer_blocks_hidden_gradients():
    rng = np.random.default_rng(2)
    params = _net(rng)
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros_like(params[-1][1]))
    x = rng.standard_normal((5, 4))
    t = rng.standard_normal((5, 5))
    y, cache = mlp.forward(params, x)
    assert np.all(y == 0)
    grads = mlp.backward(params, cache, y, t)
    for gW, gb in grads[:-1]:
        assert np.all(gW == 0) and np.all(gb == 0)
    # the output layer still learns: dW_L = g^T h_{L-1} with g = -2 t / (B K)
    assert np.allclose(grads[-1][0], (-2 * t / 25).T @ cache[-1][0], rtol=1e-13)


def test_hidden_permutation_symmetry():
    rng = np.random.default_rng(3)
    params = _net(rng)
    x = rng.standard_normal((4, 4))
    t = rng.standard_normal((4, 5))
    perm = rng.permutation(7)
    q = [list(p) for p in params]
    q[1][0] = params[1][0][perm]           # rows of layer 2 (its outputs)
    q[1][1] = params[1][1][perm]
    q[2][0] = params[2][0][:, perm]        # columns of layer 3 (its inputs)
    q = [tuple(p) for p in q]
    y0, c0 = mlp.forward(params, x)
    y1, c1 = mlp.forward(q, x)
    assert np.allclose(y0, y1, rtol=1e-13, atol=1e-14)
    g0 = mlp.backward(params, c0, y0, t)
    g1 = mlp.backward(q, c1, y1, t)
    assert np.allclose(g1[1][0], g0[1][0][perm], rtol=1e-12, atol=1e-15)
    assert np.allclose(g1[2][0], g0[2][0][:, perm], rtol=1e-12, atol=1e-15)


def test_adam_first_steps_closed_form():
    rng = np.random.default_rng(4)
    params = _net(rng, hidden=3, n_hidden=1, n_out=2)
    grads = [(rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for W, b in params]
    opt = mlp.Adam(params, lr=1e-2, eps=1e-8)
    p1 = opt.step(params, grads)
    # bias correction makes m_hat = g and v_hat = g^2 after the first step
    for (W, b), (W1, b1), (gW, gb) in zip(params, p1, grads):
        assert np.allclose(W - W1, 1e-2 * gW / (np.abs(gW) + 1e-8), rtol=1e-12)
        assert np.allclose(b - b1, 1e-2 * gb / (np.abs(gb) + 1e-8), rtol=1e-12)
    # a constant gradient keeps m_hat = g, v_hat = g^2: the same step again
    p2 = opt.step(p1, grads)
    for (W1, b1), (W2, b2), (gW, gb) in zip(p1, p2, grads):
        assert np.allclose(W1 - W2, 1e-2 * gW / (np.abs(gW) + 1e-8), rtol=1e-10)


def test_flatten_roundtrip_and_count():
    rng = np.random.default_rng(5)
    params = _net(rng, hidden=6, n_hidden=3, n_out=9)
    flat = mlp.flatten(params)
    assert flat.size == mlp.n_params(4, 6, 3, 9) == (6 * 4 + 6) + 2 * (6 * 6 + 6) + (9 * 6 + 9)
    back = mlp.unflatten(flat, 4, 6, 3, 9)
    for (W, b), (W2, b2) in zip(params, back):
        assert np.array_equal(W, W2) and np.array_equal(b, b2)
