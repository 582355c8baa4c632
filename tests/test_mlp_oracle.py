"""Pins for the FP64 reference of the sketch network (oracle/mlp.py).

* GELU at closed-form points: GELU(0) = 0, GELU'(0) = 1/2, and GELU(a) - GELU(-a) = a
  (from Phi(a) + Phi(-a) = 1); the derivative against a central difference.
* The analytic backward pass against central finite differences of the loss,
  coordinate by coordinate, on a tiny network.
* The sketch is unit length and invariant to a positive scaling of the last
  layer (W2, b2) -> (k W2, k b2); the loss is 0 when every target equals the
  sketch cosine.
"""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_closed_forms():
    a = np.array([0.0, 1.0, -1.0, 2.5, -3.0])
    g = mlp.gelu(a)
    assert g[0] == 0.0
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    assert np.allclose(mlp.gelu(a) - mlp.gelu(-a), a, atol=1e-15)
    # GELU(1) = Phi(1) = 0.5 (1 + erf(1/sqrt 2))
    assert abs(g[1] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-15
    h = 1e-6
    for x in (-2.0, -0.3, 0.7, 1.9):
        fd = (mlp.gelu(np.array([x + h]))[0] - mlp.gelu(np.array([x - h]))[0]) / (2 * h)
        assert abs(fd - mlp.gelu_grad(np.array([x]))[0]) < 1e-8


def _tiny(seed=0):
    rng = np.random.default_rng(seed)
    d, hid, out, n = 7, 5, 4, 9
    params = {k: v.astype(np.float64) for k, v in mlp.init_params(d, hid, out, seed).items()}
    params["b1"] = rng.standard_normal(hid) * 0.1
    params["b2"] = rng.standard_normal(out) * 0.1
    X = rng.standard_normal((n, d))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    P = np.array([0, 1, 2, 3, 4, 0, 7])
    Q = np.array([5, 6, 7, 8, 0, 2, 1])
    t = rng.uniform(-1, 1, len(P))
    w = rng.uniform(0.5, 2.0, len(P))
    return params, X, P, Q, t, w


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backward_matches_central_differences(seed):
    params, X, P, Q, t, w = _tiny(seed)
    grads = mlp.backward(params, X, P, Q, t, w)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2"):
        p = params[name]
        flat = p.reshape(-1)
        for idx in range(flat.size):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(params, X, P, Q, t, w)
            flat[idx] = old - h
            lm = mlp.loss(params, X, P, Q, t, w)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = grads[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 + 1e-5 * abs(fd), (name, idx, fd, an)


def test_sketch_invariances():
    params, X, P, Q, t, w = _tiny(3)
    s = mlp.forward(params, X)["s"]
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-15)
    scaled = dict(params, W2=params["W2"] * 3.0, b2=params["b2"] * 3.0)
    assert np.allclose(mlp.forward(scaled, X)["s"], s, atol=1e-14)
    c = np.sum(s[P] * s[Q], axis=1)
    assert mlp.pair_loss(s, P, Q, c, w) == 0.0
