"""Pins for the FP64 reference of the scheduler network: central finite
differences of the loss, a zero-weight closed form, and bfloat16 rounding
against hand-worked values."""
import numpy as np

from oracle import mlp


def _data(n=7, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 16))
    k = rng.integers(1, 17, n)
    prio = rng.normal(size=n)
    params = rng.normal(scale=0.3, size=mlp.NPARAMS)
    return params, x, k, prio


def test_parameter_count():
    assert mlp.NPARAMS == 6353


def test_gradient_matches_finite_differences():
    params, x, k, prio = _data()
    L, g = mlp.loss_grad(params, x, k, prio)
    assert abs(L - mlp.loss(params, x, k, prio)) < 1e-12
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(mlp.NPARAMS, 40, replace=False),
                          [0, 1023, 1024, 1087, 5183, 5184, 6270, 6335, 6352]])
    h = 1e-6
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd = (mlp.loss(p1, x, k, prio) - mlp.loss(p2, x, k, prio)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_weights_closed_form():
    # all parameters zero: uniform softmax, priority output 0
    _, x, k, prio = _data(5)
    L = mlp.loss(np.zeros(mlp.NPARAMS), x, k, prio)
    assert abs(L - (np.log(16.0) + np.mean(prio ** 2))) < 1e-12


def test_gelu_values():
    # GELU(0) = 0, GELU(z) -> z for large z, GELU(-z) = GELU(z) - z
    z = np.array([0.0, 8.0, 1.3, -1.3])
    g = mlp.gelu(z)
    assert g[0] == 0.0 and abs(g[1] - 8.0) < 1e-12
    assert abs(g[3] - (g[2] - 1.3)) < 1e-12


def test_bf16_rounding():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, -2.5, 3.14159265], np.float32)
    r = mlp.bf16_round(a)
    # 7 explicit mantissa bits (ulp(1) = 2^-7): 1 + 2^-8 is a tie -> even (1.0),
    # 1 + 3 * 2^-9 rounds up to 1 + 2^-7, 1 + 2^-9 rounds down
    assert list(r[:5]) == [1.0, 1.0, 1.0 + 2 ** -7, 1.0, -2.5]
    assert abs(r[5] - 3.140625) < 1e-7
