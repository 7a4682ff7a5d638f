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


# ---------------------------------------------------------------------------
# the bf16-operand variant
# ---------------------------------------------------------------------------

def test_bf16_rounding_fixed_points_and_ties():
    one = 1.0
    cases = {
        0.0: 0.0, one: one, -one: -one, 3.0: 3.0,
        one + 2.0 ** -8: one,                         # tie between 1 and 1 + 2^-7: even mantissa
        one + 3 * 2.0 ** -8: one + 2.0 ** -6,         # tie between 1 + 2^-7 and 1 + 2^-6: even mantissa
        one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7,  # above the tie: up
        one + 2.0 ** -9: one,                         # below the tie: down
        -(one + 3 * 2.0 ** -8): -(one + 2.0 ** -6),
        2.0 ** -130: 2.0 ** -130,                     # a subnormal float32 that bf16 holds exactly
    }
    for x, want in cases.items():
        assert mlp.bf16(np.array([x]))[0] == want, (x, mlp.bf16(np.array([x]))[0], want)


def test_bf16_rounding_agrees_with_torch():
    torch = __import__("pytest").importorskip("torch")
    x = np.random.default_rng(7).normal(scale=10.0, size=20000)
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), want)


def _grid_network(rng):
    """Weights on a 2^-4 grid and small integer inputs: every product operand
    and every hidden value the bf16 variant rounds is already a bf16 number."""
    p = {
        "W1": rng.integers(-4, 5, (64, 16)) / 16.0,
        "b1": rng.integers(-4, 5, 64) / 16.0,
        "W2": rng.integers(-2, 3, (64, 64)) / 16.0,
        "b2": rng.integers(-4, 5, 64) / 16.0,
        "w3": rng.integers(-4, 5, 64) / 16.0,
        "b3": np.asarray(0.25),
    }
    X = rng.integers(-2, 3, (50, 16)).astype(np.float64)
    return p, X


def test_bf16_forward_equals_exact_forward_when_nothing_rounds():
    rng = np.random.default_rng(8)
    p, X = _grid_network(rng)
    z1 = X @ p["W1"].T + p["b1"]
    assert np.array_equal(mlp.bf16(z1), z1)          # the construction holds
    a, _ = mlp.forward(p, X)
    b, _ = mlp.forward_bf16(p, X)
    assert np.array_equal(a, b)


def test_bf16_gradient_within_rounding_of_exact_gradient():
    # each rounded operand carries a relative error of at most 2^-9; the
    # gradient blocks are sums of products of two such operands
    rng = np.random.default_rng(9)
    p = mlp.init(11)
    X = rng.normal(size=(400, 16))
    y = (rng.random(400) < 0.3).astype(float)
    l0, g0 = mlp.loss_and_grad(mlp.quantized(p), mlp.bf16(X), y)
    l1, g1 = mlp.loss_and_grad_bf16(p, X, y)
    assert abs(l0 - l1) < 2.0 ** -8 * abs(l0)
    for k in mlp.ORDER:
        a, b = np.asarray(g0[k]).ravel(), np.asarray(g1[k]).ravel()
        assert np.linalg.norm(a - b) <= 2.0 ** -6 * np.linalg.norm(a) + 1e-12, k
