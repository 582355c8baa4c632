"""Parity of the top-1 join condition (Sec. VI-E, top-k with k = 1) with the FP64 oracle.

Every test runs ejoin_top1 through the C ABI and checks it with
parity_util.compare_top1: the rows that get a record are exactly the oracle's,
each chosen j is a best pair within 1e-5 (so it is the oracle's j wherever the
best and second best differ by more than that), and the reported similarity is
within 1e-5 of the pair's FP64 value.
"""
import os

import numpy as np
import pytest

import ejoin_inputs as inputs
import oracle
from parity_util import compare_top1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2312_01476_gb300 as pkg  # noqa: E402

PRECS = ["bf16", "tf32", "fp8"]
THREADS = os.cpu_count() or 8


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def top1(prec, R, S, selR=None, selS=None, **kw):
    with pkg.Ctx(device=0, prec=prec, **kw) as ctx:
        res = pkg.ejoin_top1(ctx, R if torch.is_tensor(R) else dev(R), S if torch.is_tensor(S) else dev(S),
                             selR, selS)
        torch.cuda.synchronize()
        st = pkg.ejoin_last_stats(ctx)
        return (res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32), res.sim.cpu().numpy(),
                st)


def clustered(n, d, k, seed, theta=0.3):
    centres = inputs.sphere_centres(k, d, seed)
    return inputs.clustered(n, d, centres, theta, seed + 1)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(300, 700, 37), (129, 1025, 128), (1000, 3000, 300), (37, 2000, 64)])
def test_top1_ragged(prec, shape):
    nR, nS, d = shape
    rng = np.random.default_rng(nR + nS + d)
    R = rng.standard_normal((nR, d)).astype(np.float32)
    S = rng.standard_normal((nS, d)).astype(np.float32)
    gi, gj, gs, st = top1(prec, R, S)
    oi, oj, os_ = oracle.top1(R, S, threads=THREADS)
    r = compare_top1(R, S, gi, gj, gs, oi, oj, os_)
    assert r["rows"] == nR and st["pairs"] == nR and st["candidates"] >= nR


@pytest.mark.parametrize("prec", PRECS)
def test_top1_clustered_near_ties(prec):
    # 20 clusters of ~150 S rows each: every row's best lies among many near-equal similarities
    d = 300
    centres = inputs.sphere_centres(20, d, 61)
    R = inputs.clustered(700, d, centres, 0.3, 62)
    S = inputs.clustered(3000, d, centres, 0.3, 63)
    gi, gj, gs, st = top1(prec, R, S)
    oi, oj, os_ = oracle.top1(R, S, threads=THREADS)
    r = compare_top1(R, S, gi, gj, gs, oi, oj, os_)
    assert r["same_j"] >= 0.95 * len(oi)


@pytest.mark.parametrize("prec", PRECS)
def test_top1_selection_both_sides(prec):
    R, S = clustered(900, 96, 10, 71), clustered(2500, 96, 10, 73)
    rng = np.random.default_rng(74)
    aR = rng.integers(0, 10, 900).astype(np.int32)
    aS = rng.integers(0, 100, 2500).astype(np.int32)
    gi, gj, gs, st = top1(prec, R, S, pkg.Sel(dev(aR), "<", 4), pkg.Sel(dev(aS), ">=", 70))
    oi, oj, os_ = oracle.top1(R, S, oracle.Selection(aR, "<", 4), oracle.Selection(aS, ">=", 70), threads=THREADS)
    compare_top1(R, S, gi, gj, gs, oi, oj, os_)
    assert st["n_sel_r"] == int((aR < 4).sum()) and st["n_sel_s"] == int((aS >= 70).sum())
    assert np.all(aS[gj] >= 70) and np.all(aR[gi] < 4)


@pytest.mark.parametrize("prec", PRECS)
def test_top1_exact_ties_go_to_the_smaller_j(prec):
    # S holds exact duplicates of some R rows at two positions; the smaller j must win, and with
    # the smaller one filtered out, the larger one
    rng = np.random.default_rng(81)
    d = 64
    R = rng.standard_normal((200, d)).astype(np.float32)
    S = rng.standard_normal((1500, d)).astype(np.float32)
    src = np.arange(0, 200, 10)
    lo = rng.choice(np.arange(0, 700), len(src), replace=False)
    hi = rng.choice(np.arange(800, 1500), len(src), replace=False)
    S[lo] = R[src]
    S[hi] = R[src]
    gi, gj, gs, st = top1(prec, R, S)
    oi, oj, os_ = oracle.top1(R, S, threads=THREADS)
    compare_top1(R, S, gi, gj, gs, oi, oj, os_)
    assert np.array_equal(gj[src], lo) and np.array_equal(oj[src], lo)
    attr = np.zeros(1500, dtype=np.int32)
    attr[lo] = 1
    gi, gj, gs, st = top1(prec, R, S, None, pkg.Sel(dev(attr), "==", 0))
    oi, oj, os_ = oracle.top1(R, S, None, oracle.Selection(attr, "==", 0), threads=THREADS)
    compare_top1(R, S, gi, gj, gs, oi, oj, os_)
    assert np.array_equal(gj[src], hi)


@pytest.mark.parametrize("prec", PRECS)
def test_top1_zero_rows_and_self_join(prec):
    rng = np.random.default_rng(91)
    X = rng.standard_normal((600, 128)).astype(np.float32)
    X[[5, 77, 300]] = 0.0  # zero rows: every similarity is 0, so the smallest j wins
    gi, gj, gs, st = top1(prec, X, X)
    oi, oj, os_ = oracle.top1(X, X, threads=THREADS)
    compare_top1(X, X, gi, gj, gs, oi, oj, os_)
    nz = np.setdiff1d(np.arange(600), [5, 77, 300])
    assert np.array_equal(gj[nz], nz)  # a non-zero row's best in a self-join is itself
    assert np.all(gj[[5, 77, 300]] == 0) and np.all(gs[[5, 77, 300]] == 0.0)


def test_top1_empty_and_unsupported():
    R, S = clustered(100, 32, 4, 95), clustered(90, 32, 4, 97)
    for prec in PRECS:
        gi, gj, gs, st = top1(prec, R[:0], S)
        assert len(gi) == 0
        gi, gj, gs, st = top1(prec, R, S[:0])
        assert len(gi) == 0
        attr = np.zeros(90, dtype=np.int32)
        gi, gj, gs, st = top1(prec, R, S, None, pkg.Sel(dev(attr), ">", 5))
        assert len(gi) == 0 and st["n_sel_s"] == 0
    with pytest.raises(pkg.EJoinError) as e:
        top1("f32", R, S)
    assert e.value.status == 7
    Rn = R.copy()
    Rn[3, 3] = np.nan
    with pytest.raises(pkg.EJoinError) as e:
        top1("bf16", Rn, S)
    assert e.value.status == 4


def test_top1_candidate_buffer_regrowth():
    # identical S rows: every column ties with the row maximum, far more candidates than the hint
    rng = np.random.default_rng(99)
    R = rng.standard_normal((300, 64)).astype(np.float32)
    S = np.repeat(rng.standard_normal((1, 64)).astype(np.float32), 2000, axis=0)
    gi, gj, gs, st = top1("bf16", R, S, capacity_hint=1024)
    assert st["contract_retries"] >= 1 and st["candidates"] == 300 * 2000
    oi, oj, os_ = oracle.top1(R, S, threads=THREADS)
    compare_top1(R, S, gi, gj, gs, oi, oj, os_)
    assert np.all(gj == 0)


@pytest.mark.parametrize("prec", PRECS)
def test_top1_full_size_sampled_rows(prec):
    # 10,000 queries x 1,000,000 rows, d = 300, the S predicate attr < 10 (10 % of S kept)
    w = inputs.topk_clustered_selection(sel_c=10, threads=THREADS)
    R, S, A = dev(w.R), dev(w.S), dev(w.attrS)
    with pkg.Ctx(device=0, prec=prec, flags=pkg.EJOIN_FLAG_TIMING) as ctx:
        res = pkg.ejoin_top1(ctx, R, S, None, pkg.Sel(A, w.opS, w.cS))
        st = pkg.ejoin_last_stats(ctx)
    assert res.count == w.R.shape[0] and st["n_sel_s"] == int((w.attrS < w.cS).sum())
    gi, gj, gs = res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32), res.sim.cpu().numpy()
    assert np.array_equal(gi, np.arange(w.R.shape[0]))
    rows = np.sort(np.random.default_rng(5).choice(w.R.shape[0], 64, replace=False))
    oi, oj, os_ = oracle.top1(w.R, w.S, None, oracle.Selection(w.attrS, w.opS, w.cS), rows=rows, threads=THREADS)
    compare_top1(w.R, w.S, gi, gj, gs, oi, oj, os_, rows=rows)
    assert np.all(w.attrS[gj] < w.cS)
    del R, S, A, res
    torch.cuda.empty_cache()
