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


def compare_top1(R, S, gi, gj, gs, oi, oj, os_, tol=1e-5, rows=None):
    """Check a GPU top-1 result (gi, gj, gs) against the oracle's (oi, oj, os_).

    The rows that get a record must be exactly the oracle's, in ascending order.
    Per row, the GPU's choice j must be a best pair within ``tol``: its FP64
    similarity is at least the oracle's maximum less ``tol`` (so where the best
    and the second best differ by more than ``tol`` it is the oracle's j), and
    the reported similarity is within ``tol`` of that FP64 value.  ``rows``:
    the R rows the oracle evaluated (the GPU records of other rows are
    ignored).  Returns a dict of statistics."""
    gi = np.asarray(gi, dtype=np.int64)
    gj = np.asarray(gj, dtype=np.int64)
    gs = np.asarray(gs, dtype=np.float64)
    assert np.all(np.diff(gi) > 0), "top-1 records are not in strictly ascending i"
    if rows is not None:
        keep = np.isin(gi, np.asarray(rows, dtype=np.int64))
        gi, gj, gs = gi[keep], gj[keep], gs[keep]
    oi = np.asarray(oi, dtype=np.int64)
    assert np.array_equal(gi, oi), f"rows with a record differ: {len(gi)} GPU vs {len(oi)} oracle"
    if len(gi) == 0:
        return {"rows": 0, "same_j": 0, "max_gap": 0.0, "max_err": 0.0}
    assert gj.max() < S.shape[0], "j out of range"
    s = oracle.sim_pairs(R, S, gi.astype(np.uint32), gj.astype(np.uint32))
    gap = np.asarray(os_, dtype=np.float64) - s
    bad = gap > tol
    assert not bad.any(), f"{bad.sum()} rows chose a j more than {tol} below the best: rows {gi[bad][:5]} " \
                          f"gap {gap[bad][:5]}"
    err = np.abs(gs - s)
    assert err.max() <= tol, f"sim error {err.max():.3g} > {tol}"
    return {"rows": int(len(gi)), "same_j": int((gj == np.asarray(oj, dtype=np.int64)).sum()),
            "max_gap": float(max(gap.max(), 0.0)), "max_err": float(err.max())}


def compare_topk(R, S, k, gi, gj, gs, oi, oj, os_, tol=1e-5, rows=None):
    """Check a GPU top-k result against the oracle's: the same rows with the same number of records
    each, in ascending i; per row, distinct columns in non-increasing reported similarity, each
    reported similarity within ``tol`` of the pair's FP64 value, and the t-th largest FP64
    similarity of the chosen columns within ``tol`` of the row's true t-th largest (so the chosen
    set is the oracle's wherever the similarities around the k-th are more than ``tol`` apart).
    Returns a dict of statistics."""
    gi = np.asarray(gi, dtype=np.int64)
    gj = np.asarray(gj, dtype=np.int64)
    gs = np.asarray(gs, dtype=np.float64)
    assert np.all(np.diff(gi) >= 0), "top-k records are not in ascending i"
    if rows is not None:
        keep = np.isin(gi, np.asarray(rows, dtype=np.int64))
        gi, gj, gs = gi[keep], gj[keep], gs[keep]
    oi = np.asarray(oi, dtype=np.int64)
    assert np.array_equal(gi, oi), f"records per row differ: {len(gi)} GPU vs {len(oi)} oracle"
    if len(gi) == 0:
        return {"rows": 0, "same_set": 0, "max_gap": 0.0, "max_err": 0.0}
    ur, cnt = np.unique(gi, return_counts=True)
    kk = int(cnt[0])
    assert np.all(cnt == kk) and kk <= k
    n = len(ur)
    J, G = gj.reshape(n, kk), gs.reshape(n, kk)
    assert J.max() < S.shape[0], "j out of range"
    assert all(len(set(r.tolist())) == kk for r in J), "a row lists a column twice"
    assert np.all(np.diff(G, axis=1) <= 0), "records of a row are not in descending similarity"
    s = oracle.sim_pairs(R, S, gi.astype(np.uint32), gj.astype(np.uint32)).reshape(n, kk)
    err = np.abs(G - s)
    assert err.max() <= tol, f"sim error {err.max():.3g} > {tol}"
    O = np.asarray(os_, dtype=np.float64).reshape(n, kk)
    gap = np.abs(np.sort(s, axis=1)[:, ::-1] - O)
    bad = gap.max(axis=1) > tol
    assert not bad.any(), f"{bad.sum()} rows chose columns outside the top {kk} by more than {tol}: rows " \
                          f"{ur[bad][:5]}"
    OJ = np.asarray(oj, dtype=np.int64).reshape(n, kk)
    same = sum(set(a.tolist()) == set(b.tolist()) for a, b in zip(J, OJ))
    return {"rows": int(n), "same_set": int(same), "max_gap": float(gap.max()), "max_err": float(err.max())}


def check_every_pair(R, S, eps, gi, gj, gs, keep_r=None, keep_s=None, sample=20000, seed=0, tol=1e-5):
    """Properties every GPU record must have, checked over the WHOLE result (at any size): ids in range
    and kept by the selections (boolean masks keep_r / keep_s), no duplicate pair, a reported similarity
    of at least eps - tol, and, on a seeded sample of the records drawn from the whole list, the FP64
    similarity within tol of the reported one and at least eps - tol.  Returns the sorted pair keys
    i * |S| + j."""
    gi = np.asarray(gi, dtype=np.int64)
    gj = np.asarray(gj, dtype=np.int64)
    gs = np.asarray(gs, dtype=np.float64)
    assert gi.size == 0 or (gi.min() >= 0 and gi.max() < R.shape[0]), "R id out of range"
    assert gj.size == 0 or (gj.min() >= 0 and gj.max() < S.shape[0]), "S id out of range"
    if keep_r is not None:
        assert np.asarray(keep_r)[gi].all(), "a pair of an R row the selection drops"
    if keep_s is not None:
        assert np.asarray(keep_s)[gj].all(), "a pair of an S row the selection drops"
    keys = np.sort(to_keys(gi, gj, S.shape[0]))
    assert keys.size < 2 or np.all(np.diff(keys) > 0), "duplicate pairs in the GPU result"
    assert gs.size == 0 or gs.min() >= float(np.float32(eps)) - tol, "a reported similarity below eps"
    if gi.size:
        idx = np.random.default_rng(seed).choice(gi.size, size=min(sample, gi.size), replace=False)
        want = oracle.sim_pairs(R, S, gi[idx].astype(np.uint32), gj[idx].astype(np.uint32))
        assert np.abs(want - gs[idx]).max() <= tol, "sampled record: reported similarity off"
        assert want.min() >= float(np.float32(eps)) - tol, "sampled record below eps in FP64"
    return keys
