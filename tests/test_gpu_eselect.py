"""Parity of the ℰ-selection scan (Sec. III-C, Eq. (ℰ-Selection)) with the FP64 oracle.

The ℰ-selection of R against a query batch Q at eps is, by definition, the
threshold join of R with the relation of queries, so the oracle is
oracle.join(R, Q, eps, selR) and the comparison rule is the join's
(parity_util.compare): identical pair sets outside |sim - eps| < 1e-5, sims
within 1e-5.  Every test calls ejoin_eselect through the C ABI.
"""
import os

import numpy as np
import pytest

import ejoin_inputs as inputs
import oracle
from parity_util import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2312_01476_gb300 as pkg  # noqa: E402

THREADS = os.cpu_count() or 8


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def esel(R, Q, eps, selR=None, capacity=None, **kw):
    with pkg.Ctx(device=0, **kw) as ctx:
        res = pkg.ejoin_eselect(ctx, R if torch.is_tensor(R) else dev(R), Q if torch.is_tensor(Q) else dev(Q), eps,
                                selR, capacity=capacity)
        torch.cuda.synchronize()
        st = pkg.ejoin_last_stats(ctx)
        return (res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32), res.sim.cpu().numpy(),
                st)


def clustered_pair(n, m, d, k, seed, theta=0.3):
    centres = inputs.sphere_centres(k, d, seed)
    return inputs.clustered(n, d, centres, theta, seed + 1), inputs.clustered(m, d, centres, theta, seed + 2)


@pytest.mark.parametrize("shape", [(1000, 1, 64), (129, 7, 300), (5000, 64, 768), (3000, 70, 128), (700, 33, 96)])
def test_eselect_matches_oracle(shape):
    # one query up to two chunks of 64; rows spanning several 128-row tiles and a ragged tail
    n, m, d = shape
    R, Q = clustered_pair(n, m, d, 10, 300 + n + m)
    eps = 0.85
    gi, gj, gs, st = esel(R, Q, eps)
    oi, oj, os_ = oracle.join(R, Q, eps, threads=THREADS)
    assert len(oi) > 0
    compare(R, Q, eps, gi, gj, gs, oi, oj, os_)
    assert st["fused"] == 1 and st["n_sel_r"] == n and st["n_sel_s"] == m


def test_eselect_selection_and_unaligned_rows_take_the_compaction_path():
    R, Q = clustered_pair(4000, 20, 300, 8, 311)
    attr = np.random.default_rng(312).integers(0, 10, 4000).astype(np.int32)
    eps = 0.85
    gi, gj, gs, st = esel(R, Q, eps, pkg.Sel(dev(attr), ">=", 7))
    oi, oj, os_ = oracle.join(R, Q, eps, oracle.Selection(attr, ">=", 7), threads=THREADS)
    compare(R, Q, eps, gi, gj, gs, oi, oj, os_)
    assert st["fused"] == 0 and st["n_sel_r"] == int((attr >= 7).sum())
    # a row stride that is not a multiple of 4 floats: read through the normalisation pass
    d = 37
    R2, Q2 = clustered_pair(1500, 9, d, 6, 313)
    wide = torch.zeros((1500, d + 1), dtype=torch.float32, device="cuda")
    wide[:, :d] = dev(R2)
    gi, gj, gs, st = esel(wide[:, :d], dev(Q2), eps)
    oi, oj, os_ = oracle.join(R2, Q2, eps, threads=THREADS)
    compare(R2, Q2, eps, gi, gj, gs, oi, oj, os_)
    assert st["fused"] == 0


def test_eselect_rows_outside_the_fp32_square_range():
    # sums of squares that overflow (rows ~1e25) or underflow (rows ~1e-25) FP32: the scan flags them and
    # the batch is repeated through the rescaling normalisation pass
    R, Q = clustered_pair(600, 5, 128, 4, 321)
    R = R.astype(np.float32)
    R[10] *= np.float32(1e25)
    R[20] *= np.float32(1e-25)
    R[30] = 0.0
    eps = 0.85
    gi, gj, gs, st = esel(R, Q, eps)
    oi, oj, os_ = oracle.join(R, Q, eps, threads=THREADS)
    compare(R, Q, eps, gi, gj, gs, oi, oj, os_)
    assert st["fused"] == 0
    assert 10 in set(oi.tolist()) and 20 in set(oi.tolist())


def test_eselect_full_filtered_product_and_regrowth():
    # eps <= -1 keeps every pair: n * m candidates, far more than the capacity hint
    R, Q = clustered_pair(2000, 40, 64, 5, 331)
    gi, gj, gs, st = esel(R, Q, -1.0, capacity=1 << 20, capacity_hint=4096)
    assert len(gi) == 2000 * 40 and st["contract_retries"] >= 1
    oi, oj, os_ = oracle.join(R, Q, -1.0, threads=THREADS)
    compare(R, Q, -1.0, gi, gj, gs, oi, oj, os_)


def test_eselect_edge_cases():
    R, Q = clustered_pair(300, 4, 64, 3, 341)
    gi, gj, gs, st = esel(R[:0], Q, 0.5)
    assert len(gi) == 0
    gi, gj, gs, st = esel(R, Q[:0], 0.5)
    assert len(gi) == 0
    gi, gj, gs, st = esel(R, Q, 1.5)  # above every similarity
    assert len(gi) == 0
    Rn = R.copy()
    Rn[7, 3] = np.nan
    with pytest.raises(pkg.EJoinError) as e:
        esel(Rn, Q, 0.5)
    assert e.value.status == 4
    Qn = Q.copy()
    Qn[1, 0] = np.inf
    with pytest.raises(pkg.EJoinError) as e:
        esel(R, Qn, 0.5)
    assert e.value.status == 4


def test_eselect_full_size_sampled_rows():
    # 10,000,000 x 768 rows (30.7 GB, generated on the device) against 32 queries at eps = 0.9, the bench
    # workload; the oracle checks 100,000 sampled rows against every query
    R, Q, eps = inputs.eselect_workload()
    with pkg.Ctx(device=0, flags=pkg.EJOIN_FLAG_TIMING) as ctx:
        res = pkg.ejoin_eselect(ctx, R, Q, eps)
        st = pkg.ejoin_last_stats(ctx)
        gi, gj, gs = (res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32),
                      res.sim.cpu().numpy())
    assert st["fused"] == 1 and res.count > 1000
    rows = np.sort(np.random.default_rng(7).choice(R.shape[0], 100_000, replace=False))
    Rs = R[torch.from_numpy(rows).cuda()].cpu().numpy()
    Qh = Q.cpu().numpy()
    oi, oj, os_ = oracle.join(Rs, Qh, eps, threads=THREADS)
    keep = np.isin(gi, rows)
    li = np.searchsorted(rows, gi[keep])
    compare(Rs, Qh, eps, li, gj[keep], gs[keep], oi, oj, os_)
    del R, Q, res
    torch.cuda.empty_cache()


@pytest.mark.parametrize("d", [4, 33, 1030])
def test_eselect_dimensions_off_the_k_slice(d):
    # the scan reads R in place with the caller's row stride (here d rounded up to 4 floats); columns past d in
    # the last 32-float K-slice read as zeros
    R, Q = clustered_pair(900, 12, d, 6, 350 + d, theta=0.2)
    ld = (d + 3) // 4 * 4
    Rw = torch.zeros((900, ld), dtype=torch.float32, device="cuda")
    Rw[:, :d] = dev(R)
    Rw[:, d:] = 7.0  # padding columns must not enter the similarity
    eps = 0.8
    gi, gj, gs, st = esel(Rw[:, :d], dev(Q), eps)
    oi, oj, os_ = oracle.join(R, Q, eps, threads=THREADS)
    compare(R, Q, eps, gi, gj, gs, oi, oj, os_)
    assert st["fused"] == 1
