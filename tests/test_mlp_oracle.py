"""Pins of the FP64 reference of the learned estimator's model (oracle/mlp.py):
its gradient against central finite differences of its own loss (an
independent derivative), and its forward pass against a network built by hand
whose output is known in closed form."""
import numpy as np

from oracle import mlp


import pytest


@pytest.mark.parametrize("absolute", [False, True])
def test_gradient_matches_finite_differences(absolute):
    rng = np.random.default_rng(0)
    n_in = 6
    p = rng.normal(0, 0.3, mlp.n_params(n_in))
    X = rng.normal(0, 1, (17, n_in))
    t = rng.normal(0, 1, 17)
    w = rng.uniform(0.5, 2.0, 17)
    _, g = mlp.loss_and_grad(p, n_in, X, t, w, absolute)
    eps = 1e-6
    idx = rng.choice(len(p), size=200, replace=False).tolist() + [len(p) - 1]
    for i in idx:
        q = p.copy(); q[i] += eps
        lp, _ = mlp.loss_and_grad(q, n_in, X, t, w, absolute)
        q[i] -= 2 * eps
        lm, _ = mlp.loss_and_grad(q, n_in, X, t, w, absolute)
        num = (lp - lm) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_forward_of_a_hand_built_network():
    # W1 copies input 0 into hidden unit 0 and -input 0 into unit 1; W2 copies
    # them to units 0 and 1; w3 = (1, 1): y = relu(x0) + relu(-x0) + b3 = |x0| + b3.
    n_in = 3
    W1 = np.zeros((n_in, 64)); W1[0, 0] = 1.0; W1[0, 1] = -1.0
    W2 = np.zeros((64, 64)); W2[0, 0] = 1.0; W2[1, 1] = 1.0
    w3 = np.zeros(64); w3[0] = w3[1] = 1.0
    p = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.25]])
    X = np.array([[2.0, 5.0, -1.0], [-3.0, 0.0, 0.0], [0.0, 1.0, 1.0]])
    np.testing.assert_allclose(mlp.forward(p, n_in, X), [2.25, 3.25, 0.25])
