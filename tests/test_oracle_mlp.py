"""Pins of the oracle's surrogate network (MLP nin -> nh -> nh -> 1, ReLU,
MSE loss, Adam) against facts that do not come from the oracle itself:
outputs of small networks worked by hand, central finite differences of the
loss, Adam's closed-form first steps, and loss decrease on a small fit.
CPU only."""
import numpy as np
import pytest

import oracle


def _random_params(nin, nh, seed, scale=0.5):
    g = np.random.default_rng(seed)
    return dict(W1=g.normal(size=(nh, nin)) * scale, b1=g.normal(size=nh) * scale,
                W2=g.normal(size=(nh, nh)) * scale / np.sqrt(nh), b2=g.normal(size=nh) * scale,
                w3=g.normal(size=nh) * scale, b3=np.array([g.normal() * scale]))


def test_forward_worked_by_hand():
    # nin = 2, nh = 2
    p = dict(W1=np.array([[1.0, -2.0], [0.5, 0.25]]), b1=np.array([0.5, -1.0]),
             W2=np.array([[2.0, -1.0], [-3.0, 1.0]]), b2=np.array([0.0, 4.0]),
             w3=np.array([1.5, -0.5]), b3=np.array([0.25]))
    # x = (1, 0.5): h1 = relu(1 - 1 + 0.5, 0.5 + 0.125 - 1) = (0.5, 0)
    #   h2 = relu(2 * 0.5 + 0, -1.5 + 4) = (1, 2.5);  y = 1.5 - 1.25 + 0.25 = 0.5
    # x = (-1, 2): h1 = relu(-1 - 4 + 0.5, -0.5 + 0.5 - 1) = (0, 0)
    #   h2 = relu(0, 4) = (0, 4);  y = -2 + 0.25 = -1.75
    y = oracle.mlp_forward(p, np.array([[1.0, 0.5], [-1.0, 2.0]]))
    assert y[0] == 0.5 and y[1] == -1.75


def test_forward_constant_when_first_layers_are_silent():
    nin, nh = 5, 7
    p = _random_params(nin, nh, 1)
    p["W2"][:] = 0.0
    p["b2"][:] = np.abs(p["b2"])
    X = np.random.default_rng(2).normal(size=(6, nin))
    y = oracle.mlp_forward(p, X)
    assert np.all(y == y[0])
    assert y[0] == pytest.approx(float(np.dot(p["w3"], p["b2"]) + p["b3"][0]), rel=1e-15)


@pytest.mark.parametrize("seed", [3, 4])
def test_gradient_matches_central_differences(seed):
    nin, nh, B = 4, 6, 5
    p = _random_params(nin, nh, seed)
    g = np.random.default_rng(seed + 100)
    X = g.normal(size=(B, nin))
    t = g.normal(size=B)
    loss, grad = oracle.mlp_loss_grad(p, X, t)
    assert loss == pytest.approx(np.mean((oracle.mlp_forward(p, X) - t) ** 2), rel=1e-14)
    h = 1e-6
    for k in oracle.MLP_KEYS:
        fd = np.zeros_like(p[k])
        for idx in np.ndindex(p[k].shape):
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += h
            lp = np.mean((oracle.mlp_forward(q, X) - t) ** 2)
            q[k][idx] -= 2 * h
            lm = np.mean((oracle.mlp_forward(q, X) - t) ** 2)
            fd[idx] = (lp - lm) / (2 * h)
        assert np.allclose(grad[k], fd, rtol=1e-5, atol=1e-8), k


def test_relu_kink_has_zero_derivative():
    # a unit whose pre-activation is exactly 0 passes no gradient
    p = dict(W1=np.array([[1.0]]), b1=np.array([-1.0]), W2=np.array([[1.0]]), b2=np.array([0.0]),
             w3=np.array([1.0]), b3=np.array([0.0]))
    _, g = oracle.mlp_loss_grad(p, np.array([[1.0]]), np.array([3.0]))
    assert g["W1"][0, 0] == 0.0 and g["W2"][0, 0] == 0.0 and g["b3"][0] == -6.0


def test_adam_first_steps_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    w = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 1e-3, 1e-8
    oracle.adam(w, g, m, v, 1, lr=lr, eps=eps)
    # bias-corrected moments equal g and g^2 after the first step
    assert np.allclose(w, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    # with the same gradient again they still do
    w2 = w.copy()
    oracle.adam(w2, g, m, v, 2, lr=lr, eps=eps)
    assert np.allclose(w2 - w, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    assert np.allclose(m, (1 - 0.9 ** 2) * g, rtol=1e-12) and np.allclose(v, (1 - 0.999 ** 2) * g * g, rtol=1e-12)


def test_adam_training_reduces_loss():
    nin, nh, B = 3, 16, 64
    p = _random_params(nin, nh, 7)
    g = np.random.default_rng(8)
    X = g.uniform(-1, 1, size=(B, nin))
    t = np.sin(X[:, 0]) + X[:, 1] * X[:, 2]
    state = {k: (np.zeros_like(p[k]), np.zeros_like(p[k])) for k in p}
    l0, _ = oracle.mlp_loss_grad(p, X, t)
    for step in range(1, 301):
        _, grad = oracle.mlp_loss_grad(p, X, t)
        for k in p:
            oracle.adam(p[k], grad[k], state[k][0], state[k][1], step, lr=1e-2)
    l1, _ = oracle.mlp_loss_grad(p, X, t)
    assert l1 < 0.2 * l0
