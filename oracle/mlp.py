"""FP64 reference of the learned sketch network (test infrastructure only).

Only tests/ and bench.py's cpu legs may import it; the CUDA path never does.

The network (the learned part of the join; the paper has none, it is the
"learned tile pruning" form of this build): for a unit-normalised embedding
row x (d values),

    a = W1 x + b1            (256)
    h = GELU(a) = a * Phi(a) = 0.5 a (1 + erf(a / sqrt 2))
    z = W2 h + b2            (64)
    s = z / ||z||            the sketch

and for a labelled pair (x_p, x_q, target t, weight w) the loss is
w (s_p . s_q - t)^2, summed over the pairs and divided by the sum of the
weights.  t is the pair's exact cosine similarity (Sec. III-A, Eq. (Cosine
Similarity)), so the sketch cosine is trained to track the true cosine.

Every function is the plain definition in float64 numpy; the backward pass
is written out by the chain rule.  Pins: tests/test_mlp_oracle.py (central
finite differences, closed-form GELU values, invariances).
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def _erf(x: np.ndarray) -> np.ndarray:
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(a: np.ndarray) -> np.ndarray:
    """Exact GELU: a * Phi(a), Phi the standard normal CDF."""
    return 0.5 * a * (1.0 + _erf(a / SQRT2))


def gelu_grad(a: np.ndarray) -> np.ndarray:
    """d/da [a Phi(a)] = Phi(a) + a phi(a)."""
    return 0.5 * (1.0 + _erf(a / SQRT2)) + a * INV_SQRT_2PI * np.exp(-0.5 * a * a)


def forward(params: dict, X: np.ndarray) -> dict:
    """Rows of X -> sketches; returns the intermediate values needed by backward."""
    W1, b1, W2, b2 = (np.asarray(params[k], dtype=np.float64) for k in ("W1", "b1", "W2", "b2"))
    X = np.asarray(X, dtype=np.float64)
    a = X @ W1.T + b1
    h = gelu(a)
    z = h @ W2.T + b2
    nz = np.sqrt(np.sum(z * z, axis=1))
    s = z / nz[:, None]
    return {"X": X, "a": a, "h": h, "z": z, "nz": nz, "s": s}


def pair_loss(s: np.ndarray, P: np.ndarray, Q: np.ndarray, t: np.ndarray, w: np.ndarray) -> float:
    """sum_k w_k (s[P_k] . s[Q_k] - t_k)^2 / sum_k w_k."""
    c = np.sum(s[P] * s[Q], axis=1)
    return float(np.sum(w * (c - t) ** 2) / np.sum(w))


def loss(params: dict, X: np.ndarray, P, Q, t, w) -> float:
    return pair_loss(forward(params, X)["s"], np.asarray(P), np.asarray(Q), np.asarray(t, np.float64),
                     np.asarray(w, np.float64))


def backward(params: dict, X: np.ndarray, P, Q, t, w) -> dict:
    """Gradients of `loss` with respect to W1, b1, W2, b2 (chain rule, float64)."""
    P = np.asarray(P)
    Q = np.asarray(Q)
    t = np.asarray(t, np.float64)
    w = np.asarray(w, np.float64)
    W2 = np.asarray(params["W2"], dtype=np.float64)
    f = forward(params, X)
    s, z, nz, a, h = f["s"], f["z"], f["nz"], f["a"], f["h"]
    c = np.sum(s[P] * s[Q], axis=1)
    g = 2.0 * w * (c - t) / np.sum(w)  # dL/dc_k
    ds = np.zeros_like(s)
    np.add.at(ds, P, g[:, None] * s[Q])
    np.add.at(ds, Q, g[:, None] * s[P])
    # s = z / |z|  ->  dz = (ds - s (s . ds)) / |z|
    dz = (ds - s * np.sum(s * ds, axis=1)[:, None]) / nz[:, None]
    dW2 = dz.T @ h
    db2 = dz.sum(axis=0)
    dh = dz @ W2
    da = dh * gelu_grad(a)
    dW1 = da.T @ f["X"]
    db1 = da.sum(axis=0)
    return {"W1": dW1, "b1": db1, "W2": dW2, "b2": db2}


def init_params(d: int, hidden: int, out: int, seed: int) -> dict:
    """Scaled Gaussian initialisation (float32 storage)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": (rng.standard_normal((hidden, d)) / math.sqrt(d)).astype(np.float32),
        "b1": np.zeros(hidden, np.float32),
        "W2": (rng.standard_normal((out, hidden)) / math.sqrt(hidden)).astype(np.float32),
        "b2": np.zeros(out, np.float32),
    }
