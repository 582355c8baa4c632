"""Test-only orchestration of the sketch training from the primitive C-ABI calls.

The library trains the sketch itself (ejoin_sketch_train: labelled set,
seeded epochs and calibration on the GPU).  This module does the same steps
from Python over the lower-level entry points (ejoin_threshold for labels,
ejoin_score_pairs, ejoin_sketch_train_step, ejoin_sketch_pair_sims), with
numpy's generator for the draws and numpy's quantile, as an independent
second route whose recall the library's must match.

Recipe: the held-out sample is joined with itself at eps - label_margin; every
pair found (matches and near misses, with their exact similarity) is a
labelled pair with weight `w_join`, and random pairs fill the set with
weight 1.  eps_sketch is the (1 - recall) quantile of the sketch cosine over
the true matches of a second held-out sample, minus a small margin.
"""
from __future__ import annotations

import numpy as np

from paper_2312_01476_gb300 import ejoin as E


def labelled_pairs(ctx: E.Ctx, X, eps: float, n_pairs: int, seed: int, label_margin: float = 0.2,
                   w_join: float = 8.0):
    """(p, q, t, w) CUDA tensors of labelled pairs over the rows of X (a held-out sample)."""
    import torch
    res = E.ejoin_threshold(ctx, X, X, eps - label_margin)
    jp, jq, jt = res.i.clone(), res.j.clone(), res.sim.clone()
    keep = jp != jq
    jp, jq, jt = jp[keep], jq[keep], jt[keep]
    n_join = min(len(jp), n_pairs // 2)
    rng = np.random.default_rng(seed)
    if len(jp) > n_join:
        sel = torch.from_numpy(rng.choice(len(jp), n_join, replace=False)).to(X.device)
        jp, jq, jt = jp[sel], jq[sel], jt[sel]
    n_rand = n_pairs - len(jp)
    rp = torch.from_numpy(rng.integers(0, X.shape[0], n_rand).astype(np.int32)).to(X.device)
    rq = torch.from_numpy(rng.integers(0, X.shape[0], n_rand).astype(np.int32)).to(X.device)
    rt = E.ejoin_score_pairs(ctx, X, X, rp, rq)
    p = torch.cat([jp, rp])
    q = torch.cat([jq, rq])
    t = torch.cat([jt, rt])
    w = torch.cat([torch.full((len(jp),), w_join, device=X.device), torch.ones(n_rand, device=X.device)])
    return p.contiguous(), q.contiguous(), t.contiguous(), w.contiguous()


def train(sk: E.Sketch, X, p, q, t, w, epochs: int = 3, batch: int = 65536, lr: float = 2e-3, seed: int = 0,
          log_every: int = 0):
    """Adam over shuffled mini-batches of the labelled pairs; returns the loss history (sampled)."""
    import torch
    inv = E.ejoin_row_inv_norm(sk.ctx, X)
    rng = np.random.default_rng(seed)
    hist = []
    n = len(p)
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(X.device)
        pp, qq, tt, ww = p[perm].contiguous(), q[perm].contiguous(), t[perm].contiguous(), w[perm].contiguous()
        for b0 in range(0, n, batch):
            b1 = min(n, b0 + batch)
            want = log_every and (b0 // batch) % log_every == 0
            loss = sk.train_step(X, inv, pp[b0:b1], qq[b0:b1], tt[b0:b1], ww[b0:b1], lr, want_loss=bool(want))
            if want:
                hist.append(loss)
    return hist


def calibrate(sk: E.Sketch, ctx: E.Ctx, X, eps: float, recall: float = 0.999, margin: float = 0.01):
    """eps_sketch such that a fraction >= recall of the true matches of X x X keep sketch cosine >= it."""
    import torch
    res = E.ejoin_threshold(ctx, X, X, eps)
    p, q = res.i.clone(), res.j.clone()
    if len(p) == 0:
        return -1.0
    inv = E.ejoin_row_inv_norm(ctx, X)
    s = sk.pair_sims(X, inv, p, q).cpu().numpy()
    return float(np.quantile(s, 1.0 - recall) - margin)
