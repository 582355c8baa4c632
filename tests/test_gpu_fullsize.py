"""Parity at the benchmark workloads' full sizes, in the launch configuration
that bench.py times, on sampled R rows the oracle computes one by one.

For each workload the GPU joins the whole relations; the FP64 oracle then
evaluates the same operator restricted to a seeded sample of (selected) R rows
against every S row, and the GPU pairs of those rows must satisfy the
comparison rule of parity_util (identical sets outside |sim - eps| < 1e-5,
similarities within 1e-5).
"""
import os

import numpy as np
import pytest

import ejoin_inputs as inputs
import oracle
from parity_util import check_every_pair, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2312_01476_gb300 as pkg  # noqa: E402

THREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def c2():
    return inputs.c2_clustered_selection(threads=THREADS)


def sampled_rows(pool, k, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(pool, size=min(k, len(pool)), replace=False))


@pytest.mark.parametrize("prec", ["bf16", "f32", "fp8", "tf32"])
def test_c2_full_size_sampled_rows(c2, prec):
    # R = 1,000,000 x S = 100,000, d = 300, attr < 100 pushed down, eps = 0.85 (the bench workload)
    w = c2
    R, S, A = (torch.from_numpy(a).cuda() for a in (w.R, w.S, w.attrR))
    with pkg.Ctx(device=0, prec=prec, flags=pkg.EJOIN_FLAG_TIMING) as ctx:
        res = pkg.ejoin_threshold(ctx, R, S, w.eps, pkg.Sel(A, w.opR, w.cR))
        st = pkg.ejoin_last_stats(ctx)
    assert st["n_sel_r"] == int((w.attrR < w.cR).sum()) and st["n_sel_s"] == w.S.shape[0]
    assert res.count == st["pairs"] and res.count > 5_000_000
    rows = sampled_rows(np.nonzero(w.attrR < w.cR)[0], 40, 2)
    oi, oj, os_ = oracle.join(w.R, w.S, w.eps, oracle.Selection(w.attrR, w.opR, w.cR), rows=rows, threads=THREADS)
    assert len(oi) > 1000
    gi, gj = res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32)
    gs = res.sim.cpu().numpy()
    compare(w.R, w.S, w.eps, gi, gj, gs, oi, oj, os_, rows=rows)
    # the whole result: ids kept by the selection, no duplicates, sims >= eps, sampled records exact
    check_every_pair(w.R, w.S, w.eps, gi, gj, gs, keep_r=w.attrR < w.cR, seed=7)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_c3_full_size_sampled_rows(prec):
    # self-join of 2,000,000 x 768 clustered rows at eps = 0.95 with the FP64 tier band 2e-3
    w = inputs.c3_clustered_selfjoin(threads=THREADS)
    X = torch.from_numpy(w.R).cuda()
    with pkg.Ctx(device=0, prec=prec, fp64_band=2e-3, flags=pkg.EJOIN_FLAG_TIMING) as ctx:
        res = pkg.ejoin_threshold(ctx, X, X, w.eps)
        st = pkg.ejoin_last_stats(ctx)
    n = w.R.shape[0]
    assert res.count >= n  # every (i, i) at sim 1
    assert st["fp64_rescored"] > 0
    rows = sampled_rows(np.arange(n), 12, 3)
    oi, oj, os_ = oracle.join(w.R, w.R, w.eps, rows=rows, threads=THREADS)
    gi, gj = res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32)
    gs = res.sim.cpu().numpy()
    compare(w.R, w.R, w.eps, gi, gj, gs, oi, oj, os_, rows=rows)
    keys = check_every_pair(w.R, w.R, w.eps, gi, gj, gs, seed=8)
    # the mirrored self-join: (j, i) present for every (i, j) (the sorted keys of the swapped pairs are
    # the same sorted keys)
    assert np.array_equal(np.sort(gj.astype(np.int64) * n + gi), keys)
    del X, res
    torch.cuda.empty_cache()


def test_c1_full_size_all_precisions():
    # 4096 x 4096, d = 128: the oracle runs in full; the expected set is exactly the 64 planted pairs
    w = inputs.c1_planted()
    oi, oj, os_ = oracle.join(w.R, w.S, w.eps, threads=THREADS)
    assert len(oi) == 64
    R, S = torch.from_numpy(w.R).cuda(), torch.from_numpy(w.S).cuda()
    for prec in ("f32", "bf16", "tf32", "fp8"):
        with pkg.Ctx(device=0, prec=prec, flags=pkg.EJOIN_FLAG_TIMING) as ctx:
            res = pkg.ejoin_threshold(ctx, R, S, w.eps)
        gi, gj = res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32)
        compare(w.R, w.S, w.eps, gi, gj, res.sim.cpu().numpy(), oi, oj, os_)
        assert set(zip(gi.tolist(), gj.tolist())) == set(zip(w.extra["pi"].tolist(), w.extra["pj"].tolist()))


def test_c4_batch_full_size_sampled_jobs():
    # 512 joins, lognormal sizes (median 20,000), d = 384, eps ~ U[0.8, 0.95], one persistent launch
    # replayed from a CUDA graph: the smallest job in full, the largest and the median job on 32 rows
    d = 384
    sizes, eps = inputs.c4_batch_sizes()
    centres = torch.from_numpy(inputs.sphere_centres(1000, d, inputs.seed_for(4))).cuda()
    jobs = []
    for k, ((nr, ns), e) in enumerate(zip(sizes.tolist(), eps.tolist())):
        R = inputs.clustered_torch(nr, d, centres, 0.3, inputs.seed_for(4) * 10000 + 2 * k)
        S = inputs.clustered_torch(ns, d, centres, 0.3, inputs.seed_for(4) * 10000 + 2 * k + 1)
        jobs.append((R, S, float(e)))
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        b = pkg.Batch(ctx, jobs, graph=True, autotune=False)
        b.run()
        b.run()  # a replay of the captured graph
        n = b.wait()
        job, gi, gj, gs = (x.cpu().numpy() for x in b.result(n))
        b.close()
    areas = sizes[:, 0] * sizes[:, 1]
    order = np.argsort(areas, kind="stable")
    for k, rows in ((int(order[0]), None), (int(order[-1]), 32), (int(order[len(order) // 2]), 32)):
        R, S, e = jobs[k]
        Rh, Sh = R.cpu().numpy(), S.cpu().numpy()
        sel = job == k
        rr = None if rows is None else sampled_rows(np.arange(len(Rh)), rows, k)
        oi, oj, os_ = oracle.join(Rh, Sh, e, rows=rr, threads=THREADS)
        compare(Rh, Sh, e, gi[sel].view(np.uint32), gj[sel].view(np.uint32), gs[sel], oi, oj, os_, rows=rr)
