"""Pins of the FP64 network oracle (CPU only): finite differences, a linear closed form, SGD/Adam."""
import numpy as np

from oracle import mlp


def _params(d, seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, mlp.n_params(d))


def test_gradient_matches_central_differences():
    d, n = 5, 17
    rng = np.random.default_rng(1)
    X = rng.normal(size=(n, d))
    t = rng.normal(size=n)
    p = _params(d, 2, 0.5)
    g = mlp.backward(p, X, t)
    h = 1e-6
    idx = rng.choice(p.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, t) - mlp.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_linear_network_gradient_is_least_squares_gradient():
    """With identity activations the net is y = A x + c with A = W3 W2 W1.  The loss gradient
    with respect to A is G = (2/N) sum_n r_n x_n^T (r = residual), so by the chain rule of a
    matrix product dL/dW1 = (W3 W2)^T G and dL/dW3 = G (W2 W1)^T + g_c (W2 b1 + b2)^T, where
    g_c = (2/N) sum_n r_n is the gradient with respect to the offset."""
    d, n = 4, 9
    rng = np.random.default_rng(3)
    X = rng.normal(size=(n, d))
    t = rng.normal(size=n)
    p = _params(d, 4)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, d)
    A = W3 @ W2 @ W1
    cvec = W3 @ (W2 @ b1 + b2) + b3
    r = (X @ A.T)[:, 0] + cvec[0] - t
    G = (2.0 / n) * (r[None, :] @ X)  # [1, d]
    gW1, gb1, gW2, gb2, gW3, gb3 = mlp.unpack(mlp.backward(p, X, t, relu=False), d)
    assert np.allclose(gW1, (W3 @ W2).T @ G, rtol=1e-12, atol=1e-14)
    g_c = (2.0 / n) * r.sum()
    assert np.allclose(gW3, G @ (W2 @ W1).T + g_c * (W2 @ b1 + b2)[None, :], rtol=1e-12, atol=1e-14)
    assert np.allclose(gb3, [(2.0 / n) * r.sum()], rtol=1e-12)
    # and the prediction itself is the affine map
    y, _ = mlp.forward(p, X, relu=False)
    assert np.allclose(y, (X @ A.T)[:, 0] + cvec[0], rtol=1e-12)


def test_training_reaches_low_loss():
    d, n = 3, 256
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(n, d))
    t = np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2]
    p = _params(d, 6, 0.4)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = mlp.loss(p, X, t)
    for step in range(1, 801):
        p, m, v = mlp.adam_step(p, mlp.backward(p, X, t), m, v, step, 3e-3)
    assert mlp.loss(p, X, t) < 0.02 * l0


def test_sgd_and_adam_first_step():
    p = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    assert np.allclose(mlp.sgd_step(p, g, 0.1), [0.95, -1.975])
    # first Adam step moves every parameter by lr * sign(g) (bias correction makes m/sqrt(v) = sign)
    q, m, v = mlp.adam_step(p, g, np.zeros(2), np.zeros(2), 1, 0.01, eps=0.0)
    assert np.allclose(q, p - 0.01 * np.sign(g))
