"""EJOIN_FLAG_SORT: records returned in ascending (i, j) order.

The oracle returns its pairs sorted lexicographically by (i, j); with the flag
the GPU result must be in that order (strictly increasing keys), hold the same
records as the unsorted call, and match the oracle under the usual parity rule.
The cases cover an odd and an even number of radix passes, a full product
whose order is known exactly, selections (original ids), a self-join, records
of more than one sort block, the host-buffer entry point and E-selection.
"""
import numpy as np
import pytest

import oracle
from parity_util import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2312_01476_gb300 as pkg  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gauss(seed, n, d):
    return np.random.default_rng(seed).standard_normal((n, d)).astype(np.float32)


def run(R, S, eps, flags, selR=None, selS=None, prec="bf16", same=False):
    with pkg.Ctx(device=0, prec=prec, flags=flags) as ctx:
        Rd = dev(R)
        res = pkg.ejoin_threshold(ctx, Rd, Rd if same else dev(S), eps, selR, selS)
        torch.cuda.synchronize()
        return (res.i.cpu().numpy().view(np.uint32).astype(np.int64),
                res.j.cpu().numpy().view(np.uint32).astype(np.int64), res.sim.cpu().numpy())


def assert_sorted_same(a, b, n_cols):
    """a: the sorted call, b: the unsorted one; same records, a in strictly increasing (i, j)."""
    ka = a[0] * n_cols + a[1]
    assert np.all(np.diff(ka) > 0), "records not in ascending (i, j) order"
    kb = b[0] * n_cols + b[1]
    ob = np.argsort(kb)
    assert np.array_equal(ka, kb[ob])
    assert np.array_equal(a[2].view(np.uint32), b[2][ob].view(np.uint32))


@pytest.mark.parametrize("shape", [(300, 200), (513, 3000)])
def test_full_product_order(shape):
    # eps = -1: every pair; the sorted result is exactly i-major, j-minor (3 and 4 radix passes)
    nR, nS = shape
    R, S = gauss(1, nR, 40), gauss(2, nS, 40)
    i, j, s = run(R, S, -1.0, pkg.EJOIN_FLAG_SORT)
    assert np.array_equal(i, np.repeat(np.arange(nR), nS))
    assert np.array_equal(j, np.tile(np.arange(nS), nR))
    want = oracle.sim_pairs(R, S, i.astype(np.uint32), j.astype(np.uint32))
    assert np.abs(s - want).max() <= 1e-5


@pytest.mark.parametrize("prec", ["bf16", "f32"])
def test_sorted_matches_oracle_order_with_selection(prec):
    rng = np.random.default_rng(3)
    R, S = gauss(4, 3000, 100), gauss(5, 1500, 100)
    aR = rng.integers(0, 1000, 3000).astype(np.int32)
    aS = rng.integers(0, 1000, 1500).astype(np.int32)
    selR, selS = pkg.Sel(dev(aR), "<", 400), pkg.Sel(dev(aS), ">=", 300)
    eps = 0.2
    a = run(R, S, eps, pkg.EJOIN_FLAG_SORT, selR, selS, prec=prec)
    b = run(R, S, eps, 0, selR, selS, prec=prec)
    assert_sorted_same(a, b, S.shape[0])
    oi, oj, os_ = oracle.join(R, S, eps, oracle.Selection(aR, "<", 400), oracle.Selection(aS, ">=", 300))
    compare(R, S, eps, a[0], a[1], a[2], oi, oj, os_)
    # pairs outside the band appear in the oracle's order
    far = np.abs(os_ - np.float32(eps)) >= 1e-5
    ko = oi[far].astype(np.int64) * S.shape[0] + oj[far]
    ka = a[0] * S.shape[0] + a[1]
    assert np.array_equal(ka[np.isin(ka, ko)], ko)


def test_sorted_self_join_and_many_blocks():
    # clustered self-join with ~1.5M records: more than one 4096-record sort block per digit
    rng = np.random.default_rng(6)
    centres = rng.standard_normal((30, 64))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    X = (centres[rng.integers(0, 30, 7000)] + 0.3 * rng.standard_normal((7000, 64)) / 8).astype(np.float32)
    eps = 0.8
    a = run(X, X, eps, pkg.EJOIN_FLAG_SORT, same=True)
    b = run(X, X, eps, 0, same=True)
    assert len(a[0]) > 1_000_000
    assert_sorted_same(a, b, X.shape[0])
    rows = np.arange(0, 7000, 700)
    oi, oj, os_ = oracle.join(X, X, eps, rows=rows)
    compare(X, X, eps, a[0], a[1], a[2], oi, oj, os_, rows=rows)


def test_sorted_host_entry_and_eselect():
    R, S = gauss(7, 2500, 64), gauss(8, 1800, 64)
    eps = 0.3
    with pkg.Ctx(device=0, prec="bf16", flags=pkg.EJOIN_FLAG_SORT) as ctx:
        pr, n = pkg.ejoin_threshold_host(ctx, R, S, eps)
        hi, hj, hs = pr["i"].astype(np.int64), pr["j"].astype(np.int64), pr["sim"].copy()
        Q = dev(S[:37])
        res = pkg.ejoin_eselect(ctx, dev(R), Q, eps)
        ei = res.i.cpu().numpy().view(np.uint32).astype(np.int64)
        ej = res.j.cpu().numpy().view(np.uint32).astype(np.int64)
    assert n > 1000 and np.all(np.diff(hi * S.shape[0] + hj) > 0)
    oi, oj, os_ = oracle.join(R, S, eps)
    compare(R, S, eps, hi, hj, hs, oi, oj, os_)
    assert len(ei) > 10 and np.all(np.diff(ei * 37 + ej) > 0)
