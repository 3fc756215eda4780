"""Pins for the oracle's plan-selection MLP (6-64-64-3, ReLU) and Adam step.

The MLP has no counterpart in the paper (which leaves access-path selection
to an optimizer, Sec. 5.2/5.3 takeaways).  The float64 oracle is held to
central finite differences, to a closed form when every ReLU is active (the
network is then affine: y = W3 (W2 (W1 x + b1) + b2) + b3, evaluated here with
numpy matrix products), and to a hand-computed Adam step.
"""
import numpy as np
import pytest

import oracle


def _unpack(p, shape):
    i, h1, h2, o = shape
    sizes = [h1 * i, h1, h2 * h1, h2, o * h2, o]
    parts, off = [], 0
    for s in sizes:
        parts.append(p[off:off + s])
        off += s
    W1, b1, W2, b2, W3, b3 = parts
    return W1.reshape(h1, i), b1, W2.reshape(h2, h1), b2, W3.reshape(o, h2), b3


def test_nparams():
    assert oracle.mlp_nparams() == 64 * 6 + 64 + 64 * 64 + 64 + 3 * 64 + 3


def test_affine_closed_form_when_all_relus_active():
    shape = oracle.MLP_SHAPE
    rng = np.random.default_rng(0)
    p = rng.uniform(0.0, 0.1, oracle.mlp_nparams())      # non-negative weights
    X = rng.uniform(0.1, 1.0, (7, 6))                       # positive inputs
    W1, b1, W2, b2, W3, b3 = _unpack(p, shape)
    want = ((X @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    T = rng.standard_normal((7, 3))
    M = np.ones((7, 3))
    Y, loss, _ = oracle.mlp(p, X, T, M)
    np.testing.assert_allclose(Y, want, rtol=1e-13, atol=1e-13)
    assert loss == pytest.approx(((want - T) ** 2).mean(), rel=1e-12)


def test_relu_clamps():
    shape = (2, 3, 3, 1)
    W1 = np.array([[1.0, 0], [-1.0, 0], [0, 1.0]])
    b1 = np.zeros(3)
    W2 = np.eye(3)
    b2 = np.zeros(3)
    W3 = np.array([[1.0, 1.0, 1.0]])
    b3 = np.zeros(1)
    p = np.concatenate([a.ravel() for a in (W1, b1, W2, b2, W3, b3)])
    Y, _, _ = oracle.mlp(p, np.array([[2.0, -5.0], [-3.0, 4.0]]), shape=shape)
    # relu(2)+relu(-2)+relu(-5) = 2 ; relu(-3)+relu(3)+relu(4) = 7
    assert list(Y[:, 0]) == [2.0, 7.0]


def test_gradient_central_differences():
    shape = oracle.MLP_SHAPE
    rng = np.random.default_rng(1)
    n = oracle.mlp_nparams()
    p = rng.standard_normal(n) * 0.3
    X = rng.standard_normal((9, 6))
    T = rng.standard_normal((9, 3))
    M = (rng.uniform(size=(9, 3)) < 0.7).astype(np.float64)
    _, loss, g = oracle.mlp(p, X, T, M, want_grad=True)
    h = 1e-6
    idx = rng.choice(n, 300, replace=False)
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp(pp, X, T, M)[1] - oracle.mlp(pm, X, T, M)[1]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_masked_entries_do_not_contribute():
    rng = np.random.default_rng(2)
    p = rng.standard_normal(oracle.mlp_nparams()) * 0.2
    X = rng.standard_normal((4, 6))
    T = rng.standard_normal((4, 3))
    M = np.zeros((4, 3))
    M[:, 1] = 1
    T2 = T.copy()
    T2[:, 0] += 100.0
    T2[:, 2] -= 50.0
    _, l1, g1 = oracle.mlp(p, X, T, M, want_grad=True)
    _, l2, g2 = oracle.mlp(p, X, T2, M, want_grad=True)
    assert l1 == l2 and np.array_equal(g1, g2)


def test_adam_step_by_hand():
    p = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m1, m2 = np.zeros(2), np.zeros(2)
    oracle.adam(p, g, m1, m2, 1, lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8)
    # first step: m_hat = g, v_hat = g^2 -> p -= lr * g/(|g|+eps) = lr * sign(g)
    np.testing.assert_allclose(p, [1.0 - 0.1 * 0.5 / (0.5 + 1e-8),
                                   -2.0 + 0.1 * 0.25 / (0.25 + 1e-8)], rtol=1e-15)
    p1 = p.copy()
    np.testing.assert_allclose(m1, [0.05, -0.025])
    np.testing.assert_allclose(m2, [0.00025, 0.0000625])
    g2 = np.array([0.1, 0.1])
    oracle.adam(p, g2, m1, m2, 2, lr=0.1)
    m1w = 0.9 * np.array([0.05, -0.025]) + 0.1 * g2
    m2w = 0.999 * np.array([0.00025, 0.0000625]) + 0.001 * g2 ** 2
    step = 0.1 * (m1w / (1 - 0.81)) / (np.sqrt(m2w / (1 - 0.999 ** 2)) + 1e-8)
    np.testing.assert_allclose(p, p1 - step, rtol=1e-12)
