"""The tolerance of the learned estimate: the fused FP32 kernel against the
FP64 oracle (oracle/mlp.py), derived from the kernel's arithmetic.

The kernel computes the features in FP32 (c_d/g exactly for a power-of-two
g; h[d]/P, log2(g)/16 and log1p(max(Eq. 11, 0))/16 each rounded once, the
last one from its own FP32 closed form), evaluates the model with FP32 fused
multiply-adds in index order (bias first), forms z = 8 y + 16 x_last and
returns expm1f(z).  A running error bound (Higham, "Accuracy and Stability of
Numerical Algorithms", Sec. 3.1: a sum of n products with one rounding each
errs by at most gamma_n * sum |terms|, gamma_n = n u / (1 - n u), u = 2^-24)
is carried through the three layers from the oracle's FP64 activations:

  E1_j = gamma_{n_in}(|b1_j| + sum_i |W1_ij x_i|) + sum_i |W1_ij| dx_i
  E2_j = gamma_64(|b2_j| + sum_i |W2_ij| (|h1_i| + E1_i)) + sum_i |W2_ij| E1_i
  Ey   = gamma_64(|b3| + sum_j |w3_j| (|h2_j| + E2_j)) + sum_j |w3_j| E2_j
  Ez   = 8 Ey + 16 dx_last + u (|z| + 8 Ey + 16 dx_last)
  |dev - oracle| <= e^z (e^Ez - 1) + 4 u |oracle|     (expm1f within 2 ulp)

(ReLU is 1-Lipschitz, so it passes errors through.)  dx_last allows the
closed form its own tolerance (1e-5 * max(|Eq. 11|, 1)) before log1p.  The
bound is a worst case; the tests also report the observed error.
"""
import numpy as np

U = 2.0 ** -24


def gamma(n):
    return n * U / (1.0 - n * U)


def learned_error_bound(p, n_in, X, plain, z, est, plain_rtol=1e-5):
    """Per-row bound on |fused kernel - oracle| for the rows the oracle did not
    send to the fallback.  X, plain, z, est: the oracle's FP64 features, closed
    form, log-space argument and estimate."""
    from oracle import mlp
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, n_in)
    X = np.asarray(X, np.float64).reshape(-1, n_in)
    plain = np.asarray(plain, np.float64)
    dx = U * np.abs(X)
    dx[:, n_in - 2] *= 2.0                                   # log2f(g) / 16
    eps_plain = plain_rtol * np.maximum(np.abs(plain), 1.0)  # the closed form's own tolerance
    base = np.log1p(np.maximum(plain, 0.0))
    dx[:, n_in - 1] = (eps_plain / (1.0 + np.maximum(plain, 0.0)) + 2 * U * base) / 16.0
    H1 = np.maximum(X @ W1 + b1, 0.0)
    E1 = gamma(n_in) * (np.abs(b1) + np.abs(X) @ np.abs(W1)) + dx @ np.abs(W1)
    H2 = np.maximum(H1 @ W2 + b2, 0.0)
    E2 = gamma(64) * (np.abs(b2) + (H1 + E1) @ np.abs(W2)) + E1 @ np.abs(W2)
    Ey = gamma(64) * (abs(b3) + (H2 + E2) @ np.abs(w3)) + E2 @ np.abs(w3)
    Ez = 8.0 * Ey + 16.0 * dx[:, n_in - 1]
    Ez = Ez + U * (np.abs(z) + Ez)
    return np.exp(z) * np.expm1(Ez) + 4 * U * np.abs(est)
