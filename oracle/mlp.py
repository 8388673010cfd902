"""Plain FP64 reference of the learned estimator's model -- TEST INFRASTRUCTURE ONLY.

The model (not in the paper; the interface is fixed by include/vate_learned.h):
y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 with hidden width 64, parameters
laid out as W1[n_in][64], b1[64], W2[64][64], b2[64], w3[64], b3, then the
gate tau (not a weight of the network: the closed form is kept where the
corrected value and the closed form are both >= tau).  Loss: mean
squared error over the rows.  Features of a host: per-age VAT counts / g, the
pool's per-age fractions, log2(g)/16, log1p(max(Eq. 11 estimate, 0))/16.
Output rule at slice close (`estimate`), in order: the closed form of Eq. 11,
flagged FALLBACK, when the host has no active VAT in the window; the closed
form, flagged FALLBACK, when the corrected value expm1(8 y + log1p(max(Eq. 11,
0))) is not a finite FP32 number; the closed form, flagged GATED, when the
corrected value and the closed form are both >= tau; otherwise that corrected
value.
Written directly from those definitions with numpy; the gradient is pinned
by finite differences, the forward pass and the output rule by hand-built
networks whose outputs are known in closed form.
"""
from __future__ import annotations

import numpy as np

HID = 64
FALLBACK = 4          # flag bit: the closed form was returned (no active VAT, or no finite correction)
GATED = 8             # flag bit: the closed form was returned (it and the corrected value are >= the gate tau)
FLT_MAX = float(np.finfo(np.float32).max)


def n_params(n_in: int) -> int:
    return n_in * HID + HID + HID * HID + HID + HID + 1 + 1      # ... b3, then the gate


def unpack(p: np.ndarray, n_in: int):
    p = np.asarray(p, np.float64)
    o = 0
    W1 = p[o:o + n_in * HID].reshape(n_in, HID); o += n_in * HID
    b1 = p[o:o + HID]; o += HID
    W2 = p[o:o + HID * HID].reshape(HID, HID); o += HID * HID
    b2 = p[o:o + HID]; o += HID
    w3 = p[o:o + HID]; o += HID
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def gate(p) -> float:
    """The gate tau: the last parameter."""
    return float(np.asarray(p, np.float64)[-1])


def forward(p, n_in, X):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in)
    X = np.asarray(X, np.float64).reshape(-1, n_in)
    H1 = np.maximum(X @ W1 + b1, 0.0)
    H2 = np.maximum(H1 @ W2 + b2, 0.0)
    return H2 @ w3 + b3


def loss_and_grad(p, n_in, X, t, w=None, absolute=False):
    """Mean (weighted) squared or absolute error over the rows and its gradient
    (same layout as p)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in)
    X = np.asarray(X, np.float64).reshape(-1, n_in)
    t = np.asarray(t, np.float64)
    n = X.shape[0]
    Z1 = X @ W1 + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2 + b2
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ w3 + b3
    e = y - t
    w = np.ones(n) if w is None else np.asarray(w, np.float64)
    if absolute:
        loss = float(np.mean(w * np.abs(e)))
        dy = w * np.sign(e) / n
    else:
        loss = float(np.mean(w * e * e))
        dy = 2.0 * w * e / n
    dw3 = H2.T @ dy
    db3 = dy.sum()
    dZ2 = np.outer(dy, w3) * (Z2 > 0)
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2.T) * (Z1 > 0)
    dW1 = X.T @ dZ1
    db1 = dZ1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3], [0.0]])   # the gate is not trained
    return loss, g


def features(o, hosts, k=None):
    """Feature rows of `hosts` from a CPU Oracle at a closed slice (window k)."""
    k = o.k if k is None else k
    ages = o.age_counts(hosts).astype(np.float64)
    hist = o.census().astype(np.float64)
    est, _, _ = o.estimate(hosts, k)
    n = len(hosts)
    X = np.zeros((n, 2 * k + 2))
    X[:, :k] = ages[:, :k] / o.g
    X[:, k:2 * k] = hist[:k] / o.P
    X[:, 2 * k] = np.log2(o.g) / 16.0
    X[:, 2 * k + 1] = np.log1p(np.maximum(est, 0.0)) / 16.0
    return X, est


def estimate(p, n_in, X, plain, k, plain_flags=None):
    """The learned estimate of each row and its flags (the closed form's
    SAT/POOLFULL bits from `plain_flags`, plus FALLBACK / GATED), by the rule
    in the module docstring.  The finiteness decision is taken in FP32, the
    precision in which the estimate is delivered."""
    X = np.asarray(X, np.float64).reshape(-1, n_in)
    plain = np.asarray(plain, np.float64)
    y = forward(p, n_in, X)
    z = 8.0 * y + np.log1p(np.maximum(plain, 0.0))
    with np.errstate(over="ignore", invalid="ignore"):
        est = np.expm1(z)
        finite32 = np.isfinite(est) & (np.abs(est) <= FLT_MAX)
    no_active = X[:, :k].sum(axis=1) == 0
    fb = no_active | ~finite32
    with np.errstate(invalid="ignore"):
        gated = ~fb & (est >= gate(p)) & (plain >= gate(p))
    out = np.where(fb | gated, plain, est)
    flags = np.zeros(len(out), np.uint8) if plain_flags is None else np.asarray(plain_flags, np.uint8).copy()
    flags[fb] |= FALLBACK
    flags[gated] |= GATED
    return out, flags, z
