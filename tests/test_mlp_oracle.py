"""Pins of the MLP oracle (CPU): the gradient is fixed by central finite
differences of the loss (a property of calculus, not a re-typed formula),
plus closed-form cases."""
import numpy as np

from oracle import mlp


def test_zero_network_closed_form():
    p = {k: np.zeros(s) for k, s in mlp.SHAPES.items()}
    X = np.random.default_rng(0).normal(size=(10, 16))
    y = np.array([0, 1] * 5)
    logit, _ = mlp.forward(p, X)
    assert np.allclose(logit, 0.0)
    assert abs(mlp.bce_loss(logit, y) - np.log(2.0)) < 1e-12
    _, g = mlp.loss_and_grad(p, X, y)
    # only the output bias sees a gradient: mean(sigmoid(0) - y) = 0.5 - 0.5
    assert abs(float(g["b3"]) - (0.5 - y.mean())) < 1e-12
    assert np.allclose(g["W1"], 0) and np.allclose(g["W2"], 0) and np.allclose(g["w3"], 0)


def test_bce_matches_naive_form():
    rng = np.random.default_rng(1)
    l = rng.normal(scale=3.0, size=100)
    y = (rng.random(100) < 0.4).astype(float)
    s = 1 / (1 + np.exp(-l))
    naive = -np.mean(y * np.log(s) + (1 - y) * np.log(1 - s))
    assert abs(mlp.bce_loss(l, y) - naive) < 1e-10


def test_gradient_by_finite_differences():
    rng = np.random.default_rng(2)
    p = mlp.init(3)
    X = rng.normal(size=(40, 16))
    y = (rng.random(40) < 0.3).astype(float)
    _, g = mlp.loss_and_grad(p, X, y)
    v = mlp.flatten(p)
    gv = mlp.flatten(g)
    idx = rng.choice(len(v), size=60, replace=False)
    h = 1e-6
    for i in idx:
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        lp = mlp.bce_loss(mlp.forward(mlp.unflatten(vp), X)[0], y)
        lm = mlp.bce_loss(mlp.forward(mlp.unflatten(vm), X)[0], y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gv[i]) < 1e-6 + 1e-5 * abs(fd), (i, fd, gv[i])


def test_adam_decreases_loss():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(256, 16))
    y = (X[:, 0] + 0.5 * X[:, 1] > 0).astype(float)
    p = mlp.init(5)
    st = {}
    l0 = mlp.loss_and_grad(p, X, y)[0]
    for _ in range(200):
        _, g = mlp.loss_and_grad(p, X, y)
        mlp.adam_step(p, g, st, lr=1e-2)
    assert mlp.loss_and_grad(p, X, y)[0] < 0.5 * l0
