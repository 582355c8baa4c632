"""The synthetic input recipes produce the distributions the workloads state."""
import math

import numpy as np

import ejoin_inputs as inputs


def _intra_fraction(theta, d=768, eps=0.95, n=1500, seed=0):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(d)
    c /= np.linalg.norm(c)
    g = np.random.default_rng(seed + 1).standard_normal((n, d))
    x = c + g * (math.tan(theta) / math.sqrt(d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    iu = np.triu_indices(n, 1)
    s = (x @ x.T)[iu]
    return float((s >= eps).mean()), float(s.mean())


def test_theta_768_gives_the_stated_match_rate():
    # bisection on theta for a 20 % intra-cluster match rate at eps = 0.95
    lo, hi = 0.05, 0.6
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        if _intra_fraction(mid)[0] > 0.2:
            lo = mid
        else:
            hi = mid
    assert abs(0.5 * (lo + hi) - inputs.THETA_768) < 1e-4
    frac, mean = _intra_fraction(inputs.THETA_768)
    assert abs(frac - 0.2) < 0.01 and abs(mean - math.cos(inputs.THETA_768) ** 2) < 2e-3


def test_clustered_rows_are_unit_and_deterministic():
    c = inputs.sphere_centres(10, 64, 5)
    a = inputs.clustered(70000, 64, c, 0.3, 6, threads=4)
    b = inputs.clustered(70000, 64, c, 0.3, 6, threads=1)
    assert np.array_equal(a, b)
    assert np.allclose(np.linalg.norm(a, axis=1), 1.0, atol=1e-5)


def test_planted_pairs_meet_the_bound():
    p = inputs.planted_gaussian(500, 400, 128, 30, 9)
    r, s = p.R[p.pi].astype(np.float64), p.S[p.pj].astype(np.float64)
    cos = np.sum(r * s, axis=1) / np.linalg.norm(r, axis=1) / np.linalg.norm(s, axis=1)
    assert cos.min() >= math.sqrt(1 - 0.09) - 1e-6


def test_batch_sizes_follow_the_recipe():
    sizes, eps = inputs.c4_batch_sizes()
    assert sizes.shape == (512, 2) and sizes.min() >= 1000 and sizes.max() <= 200000
    assert 15000 < np.median(sizes) < 25000
    assert eps.min() >= 0.8 and eps.max() <= 0.95
