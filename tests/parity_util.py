"""Comparison rule between a GPU result and the FP64 oracle.

With O the oracle's pairs and G the GPU's:
  * every (i, j) whose oracle similarity differs from eps by at least `band`
    is in both results or in neither;
  * every common pair has |sim_G - sim_O| <= tol;
  * G holds no duplicate pair.
Pairs inside the band may differ; they are counted and returned.
"""
import numpy as np

import oracle


def to_keys(i, j, n_cols):
    return np.asarray(i, dtype=np.int64) * int(n_cols) + np.asarray(j, dtype=np.int64)


def compare(R, S, eps, gi, gj, gs, oi, oj, os_, band=1e-5, tol=1e-5, rows=None):
    """Check the GPU pairs (gi, gj, gs) against the oracle's (oi, oj, os_).

    ``rows``: when the oracle ran on a sample of R rows, restrict the GPU pairs
    to those rows first.  Returns a dict of statistics."""
    gi = np.asarray(gi, dtype=np.int64)
    gj = np.asarray(gj, dtype=np.int64)
    gs = np.asarray(gs, dtype=np.float64)
    if rows is not None:
        keep = np.isin(gi, np.asarray(rows, dtype=np.int64))
        gi, gj, gs = gi[keep], gj[keep], gs[keep]
    n_cols = S.shape[0]
    gk = to_keys(gi, gj, n_cols)
    ok = to_keys(oi, oj, n_cols)
    assert len(np.unique(gk)) == len(gk), "duplicate pairs in the GPU result"
    common, g_idx, o_idx = np.intersect1d(gk, ok, assume_unique=True, return_indices=True)
    err = np.abs(gs[g_idx] - np.asarray(os_, dtype=np.float64)[o_idx]) if len(common) else np.zeros(0)
    assert err.size == 0 or err.max() <= tol, f"sim error {err.max():.3g} > {tol}"
    only_g = np.setdiff1d(gk, ok, assume_unique=True)
    only_o = np.setdiff1d(ok, gk, assume_unique=True)
    in_band = 0
    if len(only_g):
        s = oracle.sim_pairs(R, S, (only_g // n_cols).astype(np.uint32), (only_g % n_cols).astype(np.uint32))
        bad = np.abs(s - float(np.float32(eps))) >= band
        assert not bad.any(), f"{bad.sum()} GPU pairs outside the band are not oracle matches: " \
                              f"{only_g[bad][:5]} sims {s[bad][:5]}"
        in_band += len(only_g)
    if len(only_o):
        s = np.asarray(os_)[np.isin(ok, only_o)]
        bad = np.abs(s - float(np.float32(eps))) >= band
        assert not bad.any(), f"{bad.sum()} oracle pairs outside the band are missing on the GPU: " \
                              f"{only_o[bad][:5]} sims {s[bad][:5]}"
        in_band += len(only_o)
    return {"common": int(len(common)), "max_err": float(err.max()) if err.size else 0.0,
            "band_diffs": int(in_band)}
