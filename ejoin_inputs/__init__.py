"""Seeded synthetic inputs for the E-join tensor join (shared by tests, bench and smoke).

This module only draws inputs.  It holds none of the join's arithmetic (no
similarity, no threshold, no selection); the oracle and the CUDA path both
receive the arrays it returns.  Every generator is deterministic in its seed
and chunked: rows are drawn in chunks of ``CHUNK`` rows, chunk ``c`` from
``numpy.random.default_rng([seed, c])``, so any subset of chunks can be
regenerated alone and the chunks can be drawn in parallel threads.

Workload recipes (embedding shapes follow the paper's use of dense, row-major
relation matrices, Sec. IV-C; the paper's FastText/Wikipedia embeddings are not
available, so every input is synthetic):

* ``planted_gaussian``: i.i.d. N(0, 1) rows scaled to unit length, plus planted
  near-duplicate pairs S[j_k] = unit(R[i_k] + e_k) with ||e_k|| = 0.3 ||R[i_k]||.
  For any direction of e_k the angle between R[i_k] and R[i_k] + e_k is at most
  asin(0.3), so cos >= sqrt(1 - 0.09) = 0.9539 > 0.95 by construction.
* ``clustered``: unit vectors around ``n_clusters`` centres drawn uniformly on
  the sphere (normalised Gaussians); row = unit(c + g * tan(theta) / sqrt(d)),
  g ~ N(0, I), so each row sits at angle ~theta from its centre.
* ``uniform_attr``: an int32 attribute column uniform in [0, hi) for the
  pushed-down relational predicate (Sec. VI-E pre-filter).
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

CHUNK = 1 << 16


def seed_for(config: int) -> int:
    """Seed of a named workload: 1476 * 100 + config number."""
    return 1476 * 100 + int(config)


def _unit_rows(x: np.ndarray) -> np.ndarray:
    n = np.sqrt(np.einsum("ij,ij->i", x, x, dtype=np.float64))
    n[n == 0] = 1.0
    return (x / n[:, None].astype(x.dtype, copy=False)).astype(x.dtype, copy=False)


def gaussian_unit_rows(n: int, d: int, seed: int, threads: int = 8) -> np.ndarray:
    """n unit-length rows, each an i.i.d. N(0, 1) vector scaled to length 1 (float32)."""
    out = np.empty((n, d), dtype=np.float32)

    def fill(c):
        lo, hi = c * CHUNK, min(n, (c + 1) * CHUNK)
        rng = np.random.default_rng([seed, c])
        g = rng.standard_normal((hi - lo, d))
        out[lo:hi] = _unit_rows(g).astype(np.float32)

    _run_chunks(n, fill, threads)
    return out


def _run_chunks(n: int, fn, threads: int):
    n_chunks = (n + CHUNK - 1) // CHUNK
    if threads <= 1 or n_chunks <= 1:
        for c in range(n_chunks):
            fn(c)
        return
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(fn, range(n_chunks)))


@dataclass
class Planted:
    R: np.ndarray
    S: np.ndarray
    pi: np.ndarray  # planted R rows
    pj: np.ndarray  # planted S rows


def planted_gaussian(nR: int, nS: int, d: int, n_planted: int, seed: int,
                     noise_ratio: float = 0.3) -> Planted:
    """Unit Gaussian rows with ``n_planted`` near-duplicate (R, S) pairs.

    The k-th planted pair is (pi[k], pj[k]) with S[pj[k]] = unit(R[pi[k]] + e_k),
    ||e_k|| = noise_ratio * ||R[pi[k]]||, hence cos >= sqrt(1 - noise_ratio^2).
    """
    R = gaussian_unit_rows(nR, d, seed)
    S = gaussian_unit_rows(nS, d, seed + 1)
    rng = np.random.default_rng([seed, 0xFACE])
    pi = np.sort(rng.choice(nR, size=n_planted, replace=False)).astype(np.int64)
    pj = rng.choice(nS, size=n_planted, replace=False).astype(np.int64)
    e = rng.standard_normal((n_planted, d))
    r = R[pi].astype(np.float64)
    e *= (noise_ratio * np.linalg.norm(r, axis=1) / np.linalg.norm(e, axis=1))[:, None]
    S[pj] = _unit_rows(r + e).astype(np.float32)
    return Planted(R, S, pi, pj)


def sphere_centres(n_clusters: int, d: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 0xC3A7])
    return _unit_rows(rng.standard_normal((n_clusters, d))).astype(np.float32)


def clustered(n: int, d: int, centres: np.ndarray, theta: float, seed: int,
              threads: int = 8, with_ids: bool = False):
    """n unit rows, each unit(c + g * tan(theta) / sqrt(d)) around a uniformly chosen centre."""
    out = np.empty((n, d), dtype=np.float32)
    ids = np.empty(n, dtype=np.int32) if with_ids else None
    scale = np.float32(math.tan(theta) / math.sqrt(d))
    k = centres.shape[0]

    def fill(c):
        lo, hi = c * CHUNK, min(n, (c + 1) * CHUNK)
        rng = np.random.default_rng([seed, c])
        cid = rng.integers(0, k, size=hi - lo)
        g = rng.standard_normal((hi - lo, d), dtype=np.float32)
        g *= scale
        g += centres[cid]
        out[lo:hi] = _unit_rows(g)
        if ids is not None:
            ids[lo:hi] = cid

    _run_chunks(n, fill, threads)
    return (out, ids) if with_ids else out


def sketch_init_params(d: int, hidden: int, out: int, seed: int) -> np.ndarray:
    """Seeded starting parameters of the sketch network (flat layout W1, b1, W2, b2): W1 and W2 scaled
    Gaussian (1/sqrt of the fan-in), biases zero."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((hidden, d)) / math.sqrt(d)
    W2 = rng.standard_normal((out, hidden)) / math.sqrt(hidden)
    return np.concatenate([W1.ravel(), np.zeros(hidden), W2.ravel(), np.zeros(out)]).astype(np.float32)


def uniform_attr(n: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 0xA77])
    return rng.integers(0, hi, size=n, dtype=np.int32)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    R: np.ndarray
    S: np.ndarray
    eps: float
    attrR: Optional[np.ndarray] = None
    opR: str = "<"
    cR: int = 0
    attrS: Optional[np.ndarray] = None
    opS: str = "<"
    cS: int = 0
    self_join: bool = False
    extra: dict = field(default_factory=dict)


def c1_planted(scale: float = 1.0) -> Workload:
    """4096 x 4096 rows, d = 128, i.i.d. Gaussian unit rows, 64 planted pairs, eps = 0.9."""
    n = max(64, int(4096 * scale))
    p = planted_gaussian(n, n, 128, 64, seed_for(1))
    return Workload("planted-gaussian R=S=%d d=128 eps=0.9" % n, p.R, p.S, 0.9,
                    extra={"pi": p.pi, "pj": p.pj})


def c2_clustered_selection(nR: int = 1_000_000, nS: int = 100_000, d: int = 300,
                           n_clusters: int = 1000, theta: float = 0.3, eps: float = 0.85,
                           sel_c: int = 100, threads: int = 8) -> Workload:
    """Clustered unit rows (1000 centres, ~0.3 rad spread), attr ~ U[0, 1000) on R, attr < 100."""
    seed = seed_for(2)
    centres = sphere_centres(n_clusters, d, seed)
    R = clustered(nR, d, centres, theta, seed + 10, threads)
    S = clustered(nS, d, centres, theta, seed + 20, threads)
    attr = uniform_attr(nR, 1000, seed + 30)
    return Workload("clustered R=%d S=%d d=%d sel=attr<%d eps=%.2f" % (nR, nS, d, sel_c, eps),
                    R, S, eps, attrR=attr, opR="<", cR=sel_c)


# Cluster spread for the 768-d, 20,000-cluster workloads: at theta = 0.2309 rad an
# intra-cluster pair has similarity 0.9478 +- 0.0026 and reaches 0.95 with
# probability 0.20, so that the overall match rate at eps = 0.95 is 0.2 / 20,000 =
# 1e-5.  Found by bisection on theta over the pairs of one 1,500-row cluster;
# tests/test_inputs.py re-derives it.
THETA_768 = 0.23094743


def c3_clustered_selfjoin(n: int = 2_000_000, d: int = 768, n_clusters: int = 20_000, theta: float = THETA_768,
                          eps: float = 0.95, threads: int = 8) -> Workload:
    """Self-join of n clustered unit rows (20,000 tight clusters); ~1e-5 of the pairs match at eps = 0.95."""
    seed = seed_for(3)
    centres = sphere_centres(n_clusters, d, seed)
    X = clustered(n, d, centres, theta, seed + 10, threads)
    return Workload("clustered self-join n=%d d=%d clusters=%d theta=%.4f eps=%.2f" % (n, d, n_clusters, theta, eps),
                    X, X, eps, self_join=True, extra={"centres": centres, "theta": theta})


def c5_learned(n: int = 4_000_000, d: int = 768, n_clusters: int = 20_000, theta: float = THETA_768,
               eps: float = 0.9, n_heldout: int = 200_000, threads: int = 8) -> Workload:
    """4M-row clustered self-join at eps = 0.9 plus two held-out samples (training, calibration)."""
    seed = seed_for(5)
    centres = sphere_centres(n_clusters, d, seed)
    X = clustered(n, d, centres, theta, seed + 10, threads)
    Xtr = clustered(n_heldout, d, centres, theta, seed + 20, threads)
    Xcal = clustered(n_heldout, d, centres, theta, seed + 30, threads)
    return Workload("clustered self-join n=%d d=%d clusters=%d theta=%.4f eps=%.2f" % (n, d, n_clusters, theta, eps),
                    X, X, eps, self_join=True, extra={"train": Xtr, "calib": Xcal})


def topk_clustered_selection(nR: int = 10_000, nS: int = 1_000_000, d: int = 300, n_clusters: int = 1000,
                             theta: float = 0.3, sel_c: int = 100, threads: int = 8) -> Workload:
    """Top-k workload: nR query rows against nS rows (both clustered as in the c2 recipe), an int32
    attribute column attr ~ U[0, 100) on S and the pushed-down predicate attr < sel_c (sel_c percent of
    S kept; 100 keeps every row but still evaluates the predicate)."""
    seed = seed_for(6)
    centres = sphere_centres(n_clusters, d, seed)
    R = clustered(nR, d, centres, theta, seed + 10, threads)
    S = clustered(nS, d, centres, theta, seed + 20, threads)
    attr = uniform_attr(nS, 100, seed + 30)
    return Workload("top-k clustered R=%d S=%d d=%d sel=attr_S<%d" % (nR, nS, d, sel_c), R, S, float("nan"),
                    attrS=attr, opS="<", cS=sel_c)


def c4_batch_sizes(n_jobs: int = 512, median: float = 20_000, sigma: float = 1.0, lo: int = 1000,
                   hi: int = 200_000, seed: int = 0):
    """(nR, nS, eps) per job: sizes lognormal around the median, clipped to [lo, hi]; eps ~ U[0.8, 0.95]."""
    rng = np.random.default_rng([seed_for(4), seed])
    sizes = np.clip(np.round(np.exp(rng.normal(math.log(median), sigma, (n_jobs, 2)))), lo, hi).astype(np.int64)
    eps = rng.uniform(0.8, 0.95, n_jobs)
    return sizes, eps


def clustered_torch(n: int, d: int, centres, theta: float, seed: int, device="cuda"):
    """Device-side variant of `clustered` for multi-GB inputs (torch's seeded Philox generator)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    cid = torch.randint(0, centres.shape[0], (n,), generator=g, device=device)
    x = torch.randn((n, d), generator=g, device=device, dtype=torch.float32)
    x.mul_(math.tan(theta) / math.sqrt(d)).add_(centres[cid])
    x.div_(torch.linalg.vector_norm(x, dim=1, keepdim=True))
    return x


def eselect_workload(n: int = 10_000_000, d: int = 768, m: int = 32, n_clusters: int = 20_000,
                     theta: float = THETA_768, eps: float = 0.9, device="cuda"):
    """ℰ-selection workload, generated on the device: n rows clustered as in c3 (20,000 centres on
    S^(d-1), spread THETA_768) in chunks of 2^20 rows (chunk c seeded (seed + 10) * 1000 + c), and m
    query rows around the same centres (seed + 20), so that each query keeps about n / 20,000 rows at
    eps = 0.9.  Returns (R, Q, eps) as CUDA tensors and a float."""
    import torch
    seed = seed_for(7)
    centres = torch.from_numpy(sphere_centres(n_clusters, d, seed)).to(device)
    R = torch.empty((n, d), dtype=torch.float32, device=device)
    step = 1 << 20
    for c, lo in enumerate(range(0, n, step)):
        hi = min(n, lo + step)
        R[lo:hi] = clustered_torch(hi - lo, d, centres, theta, (seed + 10) * 1000 + c, device)
    Q = clustered_torch(m, d, centres, theta, seed + 20, device)
    return R, Q, eps
