"""Pins of the MLP oracle (no GPU): its chain-rule gradient against central
finite differences of its own loss, and a one-sample network small enough to
write out by hand."""
import numpy as np

from oracle import mlp


def rand_params(seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.N_PARAMS) * 0.3
    return p


def test_param_count():
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = rand_params(2)
    X = rng.standard_normal((20, 16))
    T = rng.standard_normal(20)
    L, g = mlp.grad(p, X, T)
    assert abs(L - mlp.loss(p, X, T)) < 1e-12
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, 0, 64 * 16]])  # b3, W1[0,0], b1[0]
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, T) - mlp.loss(p - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)), i


def test_one_sample_by_hand():
    # only W1[0][0] = 2, b1 = 0, W2[0][0] = 3, w3[0] = 5, b3 = 1 nonzero:
    # h1_0 = relu(2 x0), h2_0 = relu(3 h1_0), y = 5 h2_0 + 1 = 30 x0 + 1 for x0 > 0
    p = np.zeros(mlp.N_PARAMS)
    # flat offsets: W1 0..1023, b1 1024.., W2 1088.., b2 5184.., w3 5248.., b3 5312
    p[0] = 2.0
    p[1088] = 3.0
    p[5248] = 5.0
    p[-1] = 1.0
    x = np.zeros((1, 16))
    x[0, 0] = 0.5
    assert abs(mlp.forward(p, x)[0] - 16.0) < 1e-15
    L, g = mlp.grad(p, x, [10.0])
    assert abs(L - 36.0) < 1e-12
    # dL/dy = 2 (16 - 10) = 12; dL/db3 = 12; dL/dw3[0] = 12 h2_0 = 12 * 3
    assert abs(g[-1] - 12.0) < 1e-12
    assert abs(g[5248] - 36.0) < 1e-12
    # dL/dW1[0][0] = 12 * 5 * 3 * 2... = dy * w3 * W2 * x0 = 12 * 5 * 3 * 0.5
    assert abs(g[0] - 90.0) < 1e-12
    # negative input: the ReLU blocks every gradient but b3's
    x[0, 0] = -0.5
    L, g = mlp.grad(p, x, [10.0])
    assert abs(g[0]) == 0.0 and abs(g[-1] - 2 * (1.0 - 10.0)) < 1e-12
