"""Pins of the rank-model oracle (oracle/mlp.py).

Each check is a closed form, a library routine the oracle does not call, a
central-difference derivative, or a hand-computed example.
"""
import math

import numpy as np
import pytest

from oracle import mlp


def test_param_count():
    assert mlp.NPARAM == 64 * 7 + 64 + 64 * 64 + 64 + 64 + 1 == 4737


def test_bf16_round_matches_torch_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, -0.0, 1.0, -1.0, 3.0e38, 1e-30]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def test_bf16_round_ties_to_even():
    u = 2.0 ** -7                       # spacing of bfloat16 in [1, 2)
    assert mlp.bf16_round(1.0 + u / 2) == 1.0                 # tie, even is 1
    assert mlp.bf16_round(1.0 + u + u / 2) == 1.0 + 2 * u     # tie, even is 1 + 2u
    assert mlp.bf16_round(1.0 + u / 2 + 2.0 ** -20) == 1.0 + u
    assert mlp.bf16_round(-(1.0 + u / 2)) == -1.0


def _abs_network(c):
    """Parameters of y = sum_j |x_j| + c: hidden units 2j, 2j+1 carry relu(+x_j), relu(-x_j)."""
    p = np.zeros(mlp.NPARAM)
    W1 = p[:mlp.OFF_B1].reshape(64, 7)
    W2 = p[mlp.OFF_W2:mlp.OFF_B2].reshape(64, 64)
    for j in range(7):
        W1[2 * j, j] = 1.0
        W1[2 * j + 1, j] = -1.0
    for k in range(14):
        W2[k, k] = 1.0
    p[mlp.OFF_W3:mlp.OFF_W3 + 14] = 1.0
    p[mlp.OFF_B3] = c
    return p


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_closed_form(bf16):
    rng = np.random.default_rng(0)
    X = rng.integers(-64, 64, size=(50, 7)) / 8.0       # exact in bfloat16
    p = _abs_network(0.5)
    y, _ = mlp.forward(p, np.zeros(7), np.ones(7), X, bf16=bf16)
    np.testing.assert_array_equal(y, np.abs(X).sum(axis=1) + 0.5)


def test_forward_standardisation():
    X = np.array([[3.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0]])
    mean = np.array([1.0, 1.0, 0, 0, 0, 0, 0])
    std = np.array([2.0, 4.0, 1, 1, 1, 1, 1])
    y, _ = mlp.forward(_abs_network(0.0), mean, std, X)
    assert y[0] == 1.0                                    # |(3-1)/2| + |(1-1)/4|


def _random_params(rng, scale=0.3):
    return rng.standard_normal(mlp.NPARAM) * scale


def test_gradient_central_differences():
    rng = np.random.default_rng(1)
    p = _random_params(rng)
    X = rng.standard_normal((40, 7))
    t = rng.standard_normal(40)
    mean, std = np.zeros(7), np.ones(7)
    _, g = mlp.loss_grad(p, mean, std, X, t, bf16=False)
    idx = np.concatenate([rng.choice(mlp.OFF_B1, 12, replace=False),
                          mlp.OFF_B1 + rng.choice(64, 6, replace=False),
                          mlp.OFF_W2 + rng.choice(4096, 12, replace=False),
                          mlp.OFF_B2 + rng.choice(64, 6, replace=False),
                          mlp.OFF_W3 + rng.choice(64, 6, replace=False), [mlp.OFF_B3]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_grad(pp, mean, std, X, t, bf16=False)[0] -
              mlp.loss_grad(pm, mean, std, X, t, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_loss_closed_form():
    p = _abs_network(0.0)
    X = np.array([[1.0, 0, 0, 0, 0, 0, 0], [0, -2.0, 0, 0, 0, 0, 0]])
    t = np.array([0.0, 0.0])
    loss, g = mlp.loss_grad(p, np.zeros(7), np.ones(7), X, t)
    assert loss == 0.5 * (1.0 + 4.0) / 2
    assert g[mlp.OFF_B3] == (1.0 + 2.0) / 2              # mean residual


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(2)
    p = rng.standard_normal(100)
    g = rng.standard_normal(100)
    lr = 1e-3
    p1, m, v = mlp.adam_step(p, g, np.zeros(100), np.zeros(100), lr, 1)
    np.testing.assert_allclose(p1, p - lr * np.sign(g), rtol=0, atol=1e-9)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_gradient_descent_reduces_loss():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((200, 7))
    t = np.abs(X).sum(axis=1) * 0.3 + 1.0
    p = _random_params(rng, 0.2)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = mlp.loss_grad(p, np.zeros(7), np.ones(7), X, t)[0]
    for k in range(1, 301):
        _, g = mlp.loss_grad(p, np.zeros(7), np.ones(7), X, t)
        p, m, v = mlp.adam_step(p, g, m, v, 3e-3, k)
    l1 = mlp.loss_grad(p, np.zeros(7), np.ones(7), X, t)[0]
    assert l1 < 0.05 * l0


def test_node_features_hand_example():
    d = np.array([0.0, 1.0, 2.0, 3.0])
    gam = np.array([0.5, 0.25, 0.5, 0.5])
    mu = np.array([0.5, 0.75, 0.5, 0.0])
    uh = np.array([0.1, 0.2, 0.3, 0.4])
    f = mlp.node_features(d, gam, mu, uh, n=6, s0=0, s1=2)
    spread = 3.5
    # gaps 0.5, 0.25 (gamma) and 0.5, 0.75 (mu): min 0.25, lower median 0.5
    exp = [1.0, math.log10(0.25 / spread), math.log10(0.5 / spread),
           math.log10(1.5 / spread),                 # (d_2 - d_1) + gamma_2
           math.log10(0.01 + 0.04), 2.0 / 6.0, 2.0]
    np.testing.assert_allclose(f, exp, rtol=1e-14, atol=1e-15)
    # last node: no mu for the last pole, inner boundary at 2 only
    f2 = mlp.node_features(d, gam, mu, uh, n=6, s0=2, s1=4)
    assert f2[1] == pytest.approx(math.log10(0.5 / spread))
    assert f2[3] == pytest.approx(math.log10(1.5 / spread))
    # the whole merge has no inner boundary: dist = spread
    f3 = mlp.node_features(d, gam, mu, uh, n=6, s0=0, s1=4)
    assert f3[3] == 0.0
