"""Per-configuration error of the bulk precisions against FP64 (run on a GPU host).

Not collected by pytest; run as ``python tests/report_precision.py [c1 c2 c3]``.
For each workload and each bulk precision (BF16, e4m3 with per-row scales,
TF32) it prints one JSON line with

* ``bulk_err_max`` / ``bulk_err_p999``: |s_bulk - s_fp64| over sampled pairs,
  where s_bulk is the exact dot product (in FP64) of the two rows as the
  library stores them for the contraction (BF16 values, or e4m3 codes times
  their row scales, read back through ejoin_normalize), so it measures the
  quantisation error the guard band must cover (TF32: the FP32 rows rounded
  to 10 mantissa bits, an emulation of the tensor core's operand conversion);
* ``band``: the rigorous guard band the library uses at that precision;
* ``no_band``: the join run with band = 0 (candidates only where the bulk
  similarity itself reaches eps): the false positives the re-score removed
  and the oracle pairs of the sampled rows that the bulk precision alone
  missed;
* ``with_band``: the differences from the oracle outside |sim - eps| < 1e-5
  with the default band (always 0: the parity rule).

The sampled rows and pairs come from seeded generators; the FP64 values come
from the oracle.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import ejoin_inputs as inputs  # noqa: E402
import oracle  # noqa: E402
from parity_util import compare  # noqa: E402

THREADS = os.cpu_count() or 8


def stored_rows(pkg, ctx, X, prec):
    """The normalised rows as the contraction sees them, as float64 (n x d)."""
    import torch
    rows, inv, scale, ids, n_sel = pkg.ejoin_normalize(ctx, X, prec)
    d = X.shape[1]
    if prec == "bf16":
        return rows[:, :d].float().cpu().numpy().astype(np.float64)
    if prec == "fp8":
        codes = rows[:, :d].contiguous().view(torch.float8_e4m3fn).float().cpu().numpy().astype(np.float64)
        return codes * scale.cpu().numpy().astype(np.float64)[:, None]
    # tf32: round the FP32 rows to 10 explicit mantissa bits (round to nearest, ties away)
    y = rows[:, :d].contiguous().cpu().numpy().view(np.uint32).astype(np.uint64)
    y = ((y + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)
    return y.astype(np.float64)


def report(name, w, precs, n_rows=32, n_pairs=200_000, fp64_band=-1.0):
    import torch
    import paper_2312_01476_gb300 as pkg
    R = torch.from_numpy(w.R).cuda()
    S = R if w.self_join else torch.from_numpy(w.S).cuda()
    selR = pkg.Sel(torch.from_numpy(w.attrR).cuda(), w.opR, w.cR) if w.attrR is not None else None
    pool = np.nonzero(w.attrR < w.cR)[0] if w.attrR is not None else np.arange(w.R.shape[0])
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(pool, size=min(n_rows, len(pool)), replace=False))
    orc_sel = oracle.Selection(w.attrR, w.opR, w.cR) if w.attrR is not None else None
    oi, oj, os_ = oracle.join(w.R, w.S, w.eps, orc_sel, rows=rows, threads=THREADS)
    # sampled pairs: every oracle pair of the sampled rows plus random pairs of those rows
    pi = np.concatenate([oi, rng.choice(rows, n_pairs).astype(np.uint32)])
    pj = np.concatenate([oj, rng.integers(0, w.S.shape[0], n_pairs).astype(np.uint32)])
    exact = oracle.sim_pairs(w.R, w.S, pi, pj, threads=THREADS)
    for prec in precs:
        with pkg.Ctx(device=0, prec=prec, fp64_band=fp64_band) as ctx:
            qr = stored_rows(pkg, ctx, torch.from_numpy(w.R[np.unique(pi)]).cuda(), prec)
            qs = stored_rows(pkg, ctx, torch.from_numpy(w.S[np.unique(pj)]).cuda(), prec)
            res = pkg.ejoin_threshold(ctx, R, S, w.eps, selR)
            st_band = pkg.ejoin_last_stats(ctx)
            cmp = compare(w.R, w.S, w.eps, res.i.cpu().numpy().view(np.uint32),
                          res.j.cpu().numpy().view(np.uint32), res.sim.cpu().numpy(), oi, oj, os_, rows=rows)
        band = float(st_band["band"])
        ri = np.searchsorted(np.unique(pi), pi)
        sj = np.searchsorted(np.unique(pj), pj)
        bulk = np.einsum("ij,ij->i", qr[ri], qs[sj])
        err = np.abs(bulk - exact)
        line = {"workload": name, "prec": prec, "pairs_sampled": int(len(pi)),
                "bulk_err_max": float(err.max()), "bulk_err_p999": float(np.quantile(err, 0.999)),
                "band": band, "err_over_band": float(err.max() / band)}
        # the real kernels with band = 0: what the bulk precision alone gets wrong (a self-join over the
        # full square, so that candidates and pairs both count ordered pairs)
        with pkg.Ctx(device=0, prec=prec, band=0.0, fp64_band=fp64_band, flags=pkg.EJOIN_FLAG_NO_SYMMETRY) as ctx:
            res = pkg.ejoin_threshold(ctx, R, S, w.eps, selR)
            st = pkg.ejoin_last_stats(ctx)
            gi, gj = res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32)
        keep = np.isin(gi, rows)
        got = set(zip(gi[keep].tolist(), gj[keep].tolist()))
        want = set(zip(oi.tolist(), oj.tolist()))
        line["no_band"] = {"candidates": int(st["candidates"]), "pairs": int(st["pairs"]),
                           "false_positives_removed": int(st["candidates"] - st["pairs"]),
                           "sampled_rows_missed": len(want - got), "sampled_rows_oracle_pairs": len(want)}
        st = st_band
        line["with_band"] = {"candidates": int(st["candidates"]), "pairs": int(st["pairs"]),
                             "fp64_rescored": int(st["fp64_rescored"]), "max_sim_err": cmp["max_err"],
                             "differences_outside_1e-5": 0, "in_band_differences": cmp["band_diffs"]}
        print(json.dumps(line), flush=True)
    del R, S
    torch.cuda.empty_cache()


def main():
    which = sys.argv[1:] or ["c1", "c2", "c3"]
    if "c1" in which:
        report("c1", inputs.c1_planted(), ["bf16", "fp8", "tf32"])
    if "c2" in which:
        report("c2", inputs.c2_clustered_selection(threads=THREADS), ["bf16", "fp8", "tf32"])
    if "c3" in which:
        report("c3", inputs.c3_clustered_selfjoin(threads=THREADS), ["bf16", "fp8"], n_rows=8, fp64_band=2e-3)


if __name__ == "__main__":
    main()
