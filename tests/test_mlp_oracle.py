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
    p = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.25], [np.inf]])
    X = np.array([[2.0, 5.0, -1.0], [-3.0, 0.0, 0.0], [0.0, 1.0, 1.0]])
    np.testing.assert_allclose(mlp.forward(p, n_in, X), [2.25, 3.25, 0.25])


def _abs_net(n_in, b3, tau=np.inf):
    # y = relu(x0) + relu(-x0) + b3 = |x0| + b3 (as in the forward pin); gate tau
    W1 = np.zeros((n_in, 64)); W1[0, 0] = 1.0; W1[0, 1] = -1.0
    W2 = np.zeros((64, 64)); W2[0, 0] = 1.0; W2[1, 1] = 1.0
    w3 = np.zeros(64); w3[0] = w3[1] = 1.0
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [b3], [tau]])


def test_learned_output_of_a_hand_built_network():
    # k = 2, n_in = 6: columns 0-1 are per-age counts / g.  y = |x0| + 0.25;
    # z = 8 y + log1p(max(plain, 0)).
    k, n_in = 2, 6
    p = _abs_net(n_in, 0.25)
    X = np.array([[0.5, 0.0, 0, 0, 0.75, 0.1],      # y = 0.75, plain = e^2 - 1: z = 6 + 2
                  [0.125, 0.25, 0, 0, 0.75, 0.1],   # y = 0.375, plain negative: z = 3 + 0
                  [0.0, 0.5, 0, 0, 0.75, 0.1]])     # y = 0.25, plain = 0: z = 2
    plain = np.array([np.expm1(2.0), -7.5, 0.0])
    est, fl, z = mlp.estimate(p, n_in, X, plain, k, np.array([1, 0, 2], np.uint8))
    np.testing.assert_allclose(z, [8.0, 3.0, 2.0], rtol=1e-15)
    np.testing.assert_allclose(est, [np.expm1(8.0), np.expm1(3.0), np.expm1(2.0)], rtol=1e-15)
    np.testing.assert_array_equal(fl, [1, 0, 2])          # closed form's flags kept, no fallback


def test_learned_output_zero_model_reproduces_the_clamped_closed_form():
    # a model that outputs 0 everywhere returns max(Eq. 11, 0) (up to the
    # expm1(log1p(.)) round trip)
    k, n_in = 3, 8
    p = np.zeros(mlp.n_params(n_in))
    p[-1] = np.inf                                        # no gate
    rng = np.random.default_rng(4)
    X = rng.uniform(0.01, 1, (50, n_in))
    plain = rng.normal(0, 300, 50)
    est, fl, _ = mlp.estimate(p, n_in, X, plain, k)
    np.testing.assert_allclose(est, np.maximum(plain, 0.0), rtol=1e-13, atol=1e-12)
    assert not fl.any()


def test_learned_output_falls_back_to_the_closed_form():
    k, n_in = 2, 6
    p = _abs_net(n_in, 0.0)
    X = np.array([[0.0, 0.0, 0, 0, 0.75, 0.1],     # no active VAT: per-age counts all 0
                  [-12.0, 0.01, 0, 0, 0.75, 0.1],  # y = 12: z = 96 > ln(FLT_MAX) = 88.72
                  [-11.0, 0.01, 0, 0, 0.75, 0.1],  # y = 11: z = 88, finite in FP32
                  [0.0, 0.125, 0, 0, 0.75, 0.1]])  # active VATs, y = 0
    plain = np.array([3.5, 100.0, 0.0, 41.0])
    est, fl, _ = mlp.estimate(p, n_in, X, plain, k, np.array([0, 1, 0, 0], np.uint8))
    assert est[0] == 3.5 and fl[0] == mlp.FALLBACK
    assert est[1] == 100.0 and fl[1] == 1 | mlp.FALLBACK
    assert np.isclose(est[2], np.expm1(88.0), rtol=1e-15) and fl[2] == 0
    assert np.isclose(est[3], 41.0, rtol=1e-13) and fl[3] == 0


def test_learned_output_gate_returns_the_closed_form_where_both_are_above_tau():
    # tau = 100: where the corrected value expm1(8 y + log1p(plain)) and the
    # closed form are both >= 100 the closed form is kept (GATED); where only
    # one of them is (row 2: the corrected value; the second net: the closed
    # form), the corrected value; a host with no active VAT is FALLBACK
    k, n_in = 2, 6
    p = _abs_net(n_in, 0.25, tau=100.0)           # y = |x0| + 0.25
    X = np.array([[0.25, 0.1, 0, 0, 0.75, 0.1],     # y = 0.5:  z = 4 + 0.5 = 4.5, e = 89
                  [0.5, 0.0, 0, 0, 0.75, 0.1],      # y = 0.75: z = 6 + log1p(3000)
                  [0.0, 0.25, 0, 0, 0.75, 0.1],     # y = 0.25: z = 2 + 3 = 5, e = 147, closed form 19
                  [0.0, 0.0, 0, 0, 0.75, 0.1]])     # no active VAT
    plain = np.array([np.expm1(0.5), 3000.0, np.expm1(3.0), 500.0])
    est, fl, z = mlp.estimate(p, n_in, X, plain, k)
    np.testing.assert_allclose(z[[0, 2]], [4.5, 5.0], rtol=1e-15)
    assert np.isclose(est[0], np.expm1(4.5), rtol=1e-15) and fl[0] == 0
    assert est[1] == 3000.0 and fl[1] == mlp.GATED
    assert np.isclose(est[2], np.expm1(5.0), rtol=1e-15) and fl[2] == 0
    assert est[3] == 500.0 and fl[3] == mlp.FALLBACK
    # y = |x0| - 0.5 = -0.5: a closed form of 500 corrected to 501 e^-4 - 1 = 8.2, below tau: not gated
    q = _abs_net(n_in, -0.5, tau=100.0)
    est, fl, z = mlp.estimate(q, n_in, np.array([[0.0, 0.25, 0, 0, 0.75, 0.1]]), np.array([500.0]), k)
    assert np.isclose(z[0], np.log(501.0) - 4.0, rtol=1e-15)
    assert np.isclose(est[0], 501.0 * np.exp(-4.0) - 1.0, rtol=1e-13) and fl[0] == 0


def test_gradient_of_the_gate_is_zero():
    rng = np.random.default_rng(9)
    n_in = 4
    p = rng.normal(0, 0.3, mlp.n_params(n_in))
    _, g = mlp.loss_and_grad(p, n_in, rng.normal(0, 1, (9, n_in)), rng.normal(0, 1, 9))
    assert g.shape == p.shape and g[-1] == 0.0
