"""Parity of the top-k join condition (Sec. VI-E; k up to 32) with the FP64 oracle.

Every test runs ejoin_topk through the C ABI and checks it with
parity_util.compare_topk: the same rows with min(k, kept S rows) records each,
distinct columns in descending similarity, similarities within 1e-5 of FP64,
and the chosen columns' FP64 similarities within 1e-5 of the row's true top k.
"""
import os

import numpy as np
import pytest

import ejoin_inputs as inputs
import oracle
from parity_util import compare_topk

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2312_01476_gb300 as pkg  # noqa: E402

PRECS = ["bf16", "tf32", "fp8"]
THREADS = os.cpu_count() or 8


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def topk(prec, R, S, k, selR=None, selS=None, **kw):
    with pkg.Ctx(device=0, prec=prec, **kw) as ctx:
        res = pkg.ejoin_topk(ctx, R if torch.is_tensor(R) else dev(R), S if torch.is_tensor(S) else dev(S), k,
                             selR, selS)
        torch.cuda.synchronize()
        st = pkg.ejoin_last_stats(ctx)
        return (res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32), res.sim.cpu().numpy(),
                st)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape,k", [((300, 5000, 37), 2), ((129, 9000, 128), 7), ((1000, 6000, 300), 32),
                                     ((37, 4100, 64), 32), ((64, 300, 96), 32)])
def test_topk_ragged(prec, shape, k):
    # (64, 300): two column groups for k = 32, so every column is a candidate
    nR, nS, d = shape
    rng = np.random.default_rng(nR + nS + d + k)
    R = rng.standard_normal((nR, d)).astype(np.float32)
    S = rng.standard_normal((nS, d)).astype(np.float32)
    gi, gj, gs, st = topk(prec, R, S, k)
    oi, oj, os_ = oracle.topk(R, S, k, threads=THREADS)
    r = compare_topk(R, S, k, gi, gj, gs, oi, oj, os_)
    assert r["rows"] == nR and st["pairs"] == nR * k and st["candidates"] >= nR * k


@pytest.mark.parametrize("prec", PRECS)
def test_topk_clustered_near_ties(prec):
    d = 300
    centres = inputs.sphere_centres(20, d, 161)
    R = inputs.clustered(500, d, centres, 0.3, 162)
    S = inputs.clustered(6000, d, centres, 0.3, 163)
    gi, gj, gs, st = topk(prec, R, S, 32)
    oi, oj, os_ = oracle.topk(R, S, 32, threads=THREADS)
    r = compare_topk(R, S, 32, gi, gj, gs, oi, oj, os_)
    assert r["same_set"] >= 0.5 * r["rows"]


@pytest.mark.parametrize("prec", PRECS)
def test_topk_selection_and_short_s(prec):
    rng = np.random.default_rng(171)
    R = rng.standard_normal((700, 80)).astype(np.float32)
    S = rng.standard_normal((5000, 80)).astype(np.float32)
    aR = rng.integers(0, 10, 700).astype(np.int32)
    aS = rng.integers(0, 1000, 5000).astype(np.int32)
    for cS, k in ((300, 16), (3, 16)):  # about 1500 kept S rows; then about 15, fewer than k
        gi, gj, gs, st = topk(prec, R, S, k, pkg.Sel(dev(aR), "<", 6), pkg.Sel(dev(aS), "<", cS))
        oi, oj, os_ = oracle.topk(R, S, k, oracle.Selection(aR, "<", 6), oracle.Selection(aS, "<", cS),
                                  threads=THREADS)
        compare_topk(R, S, k, gi, gj, gs, oi, oj, os_)
        kk = min(k, int((aS < cS).sum()))
        assert st["pairs"] == int((aR < 6).sum()) * kk
        assert np.all(aS[gj] < cS) and np.all(aR[gi] < 6)


@pytest.mark.parametrize("prec", PRECS)
def test_topk_exact_ties_at_the_boundary(prec):
    # S holds three exact copies of R[src] at increasing positions; with k = 2 the two smaller j win
    rng = np.random.default_rng(181)
    d = 64
    R = rng.standard_normal((120, d)).astype(np.float32)
    S = rng.standard_normal((3000, d)).astype(np.float32)
    src = np.arange(0, 120, 6)
    pos = np.sort(rng.choice(3000, (len(src), 3), replace=False).reshape(len(src), 3), axis=1)
    for t in range(3):
        S[pos[:, t]] = R[src]
    gi, gj, gs, st = topk(prec, R, S, 2)
    oi, oj, os_ = oracle.topk(R, S, 2, threads=THREADS)
    compare_topk(R, S, 2, gi, gj, gs, oi, oj, os_)
    J = gj.reshape(120, 2)
    assert np.array_equal(J[src], pos[:, :2]) and np.array_equal(oj.reshape(120, 2)[src], pos[:, :2])


def test_topk_wide_column_groups():
    # 2,200,000 S rows: more than 8192 groups of 256 columns, so pass 0 widens the groups to 512
    rng = np.random.default_rng(191)
    d = 32
    R = rng.standard_normal((300, d)).astype(np.float32)
    S = rng.standard_normal((2_200_000, d)).astype(np.float32)
    gi, gj, gs, st = topk("bf16", R, S, 32)
    rows = np.sort(rng.choice(300, 24, replace=False))
    oi, oj, os_ = oracle.topk(R, S, 32, rows=rows, threads=THREADS)
    compare_topk(R, S, 32, gi, gj, gs, oi, oj, os_, rows=rows)


@pytest.mark.parametrize("order", ["shuffled", "sorted_by_cluster"])
def test_topk_sampled_first_pass(order):
    # 300,000 S rows = 1172 column tiles: the first pass samples every 8th tile (k = 32 needs >= 128);
    # with S sorted by cluster a row's neighbours sit in a few consecutive tiles the sample may miss,
    # which loosens the threshold but must not change the result
    d = 64
    centres = inputs.sphere_centres(300, d, 201)
    R = inputs.clustered(200, d, centres, 0.3, 202)
    S, cid = inputs.clustered(300_000, d, centres, 0.3, 203, with_ids=True)
    if order == "sorted_by_cluster":
        S = np.ascontiguousarray(S[np.argsort(cid, kind="stable")])
    for prec in PRECS:
        gi, gj, gs, st = topk(prec, R, S, 32)
        rows = np.arange(0, 200, 5)
        oi, oj, os_ = oracle.topk(R, S, 32, rows=rows, threads=THREADS)
        compare_topk(R, S, 32, gi, gj, gs, oi, oj, os_, rows=rows)
        assert st["pairs"] == 200 * 32


def test_topk_regrowth_and_invalid_k():
    rng = np.random.default_rng(199)
    R = rng.standard_normal((200, 64)).astype(np.float32)
    S = np.repeat(rng.standard_normal((1, 64)).astype(np.float32), 1500, axis=0)
    gi, gj, gs, st = topk("bf16", R, S, 5, capacity_hint=1024)
    assert st["contract_retries"] >= 1 and st["candidates"] == 200 * 1500
    oi, oj, os_ = oracle.topk(R, S, 5, threads=THREADS)
    compare_topk(R, S, 5, gi, gj, gs, oi, oj, os_)
    assert np.all(gj.reshape(200, 5) == np.arange(5))
    for k in (0, 33):
        with pytest.raises(pkg.EJoinError) as e:
            topk("bf16", R, S, k)
        assert e.value.status == 1


@pytest.mark.parametrize("prec", PRECS)
def test_topk_full_size_sampled_rows(prec):
    # 10,000 queries x 1,000,000 rows, d = 300, k = 32, the S predicate attr < 50 (half of S kept)
    w = inputs.topk_clustered_selection(sel_c=50, threads=THREADS)
    R, S, A = dev(w.R), dev(w.S), dev(w.attrS)
    with pkg.Ctx(device=0, prec=prec, flags=pkg.EJOIN_FLAG_TIMING) as ctx:
        res = pkg.ejoin_topk(ctx, R, S, 32, None, pkg.Sel(A, w.opS, w.cS))
        st = pkg.ejoin_last_stats(ctx)
    assert res.count == 32 * w.R.shape[0] and st["n_sel_s"] == int((w.attrS < w.cS).sum())
    gi, gj, gs = res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32), res.sim.cpu().numpy()
    rows = np.sort(np.random.default_rng(6).choice(w.R.shape[0], 48, replace=False))
    oi, oj, os_ = oracle.topk(w.R, w.S, 32, None, oracle.Selection(w.attrS, w.opS, w.cS), rows=rows,
                              threads=THREADS)
    compare_topk(w.R, w.S, 32, gi, gj, gs, oi, oj, os_, rows=rows)
    assert np.all(w.attrS[gj] < w.cS)
    del R, S, A, res
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d", [4, 1030])
def test_topk_small_and_large_dimensions(prec, d):
    rng = np.random.default_rng(211 + d)
    R = rng.standard_normal((200, d)).astype(np.float32)
    S = rng.standard_normal((2500, d)).astype(np.float32)
    gi, gj, gs, st = topk(prec, R, S, 8)
    oi, oj, os_ = oracle.topk(R, S, 8, threads=THREADS)
    compare_topk(R, S, 8, gi, gj, gs, oi, oj, os_)
