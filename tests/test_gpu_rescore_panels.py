"""The panel-ordered re-score against the emission-order re-score and the oracle.

By default the threshold join buckets its candidates by panels of consecutive
R rows and stages each panel's FP32 rows in shared memory; EJOIN_FLAG_GATHER_RESCORE
keeps the emission-order kernel, which gathers both rows of every candidate.
Per candidate both evaluate the same FP32 dot product in the same order, so the
two must return the same pairs with bit-identical similarities.  The cases
cover every row-width class of the kernels (d = 4 ... 1024), ragged panel
tails, selections on both sides (operand rows mapped to original ids), the
mirrored self-join, panels cut into many chunks (eps = -1), the accurate tier
(a wide FP64 band) and the shapes that fall back to the emission-order kernel.
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
from paper_2312_01476_gb300 import ejoin as E  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def clustered(seed, n, d, centres, spread):
    """Rows at about `spread` rad around unit centres, scaled by random norms."""
    rng = np.random.default_rng(seed)
    c = centres[rng.integers(0, len(centres), n)]
    c = c / np.linalg.norm(c, axis=1, keepdims=True)
    x = c + rng.standard_normal((n, d)) * (spread / np.sqrt(d))
    return (x * rng.uniform(0.5, 3.0, (n, 1))).astype(np.float32)


def joined(prec, R, S, eps, flags=0, selR=None, selS=None, **kw):
    # these joins are below the size where the panel order is the default: ask for it unless gathering
    if not flags & pkg.EJOIN_FLAG_GATHER_RESCORE:
        flags |= pkg.EJOIN_FLAG_PANEL_RESCORE
    with pkg.Ctx(device=0, prec=prec, flags=flags, **kw) as ctx:
        Rd = dev(R)
        Sd = Rd if S is R else dev(S)
        res = pkg.ejoin_threshold(ctx, Rd, Sd, eps, selR, selS)
        torch.cuda.synchronize()
        st = pkg.ejoin_last_stats(ctx)
    i = res.i.cpu().numpy().view(np.uint32).astype(np.int64)
    j = res.j.cpu().numpy().view(np.uint32).astype(np.int64)
    s = res.sim.cpu().numpy()
    order = np.lexsort((j, i))
    return i[order], j[order], s[order], st


def same_bits(a, b):
    ai, aj, asim, _ = a
    bi, bj, bsim, _ = b
    assert np.array_equal(ai, bi) and np.array_equal(aj, bj), "pair sets differ"
    assert np.array_equal(asim.view(np.uint32), bsim.view(np.uint32)), "similarities differ in some bit"


@pytest.mark.parametrize("d", [4, 64, 128, 200, 300, 384, 480, 768, 1024])
def test_panels_equal_gathers_and_oracle(d):
    rng = np.random.default_rng(d)
    centres = rng.standard_normal((40, d))
    # R rows not a multiple of any panel height; clusters give many candidates per row
    R = clustered(d + 1, 1000 + d % 97, d, centres, 0.6)
    S = clustered(d + 2, 1500 - d % 89, d, centres, 0.6)
    eps = 0.6
    a = joined("bf16", R, S, eps)
    b = joined("bf16", R, S, eps, flags=E.EJOIN_FLAG_GATHER_RESCORE)
    same_bits(a, b)
    assert len(a[0]) > 5000
    oi, oj, os_ = oracle.join(R, S, eps)
    compare(R, S, eps, a[0], a[1], a[2], oi, oj, os_)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "tf32", "f32"])
def test_panels_with_selection_and_self_join(prec):
    d = 96
    rng = np.random.default_rng(5)
    centres = rng.standard_normal((30, d))
    R = clustered(6, 2300, d, centres, 0.5)
    S = clustered(7, 1700, d, centres, 0.5)
    aR = rng.integers(0, 10, len(R)).astype(np.int32)
    aS = rng.integers(0, 10, len(S)).astype(np.int32)
    selR, selS = pkg.Sel(dev(aR), "<", 6), pkg.Sel(dev(aS), "!=", 3)
    eps = 0.7
    a = joined(prec, R, S, eps, selR=selR, selS=selS)
    b = joined(prec, R, S, eps, flags=E.EJOIN_FLAG_GATHER_RESCORE, selR=selR, selS=selS)
    same_bits(a, b)
    oi, oj, os_ = oracle.join(R, S, eps, oracle.Selection(aR, "<", 6), oracle.Selection(aS, "!=", 3))
    compare(R, S, eps, a[0], a[1], a[2], oi, oj, os_)
    # self-join: the tensor-core precisions contract the upper triangle and mirror in the re-score
    a = joined(prec, R, R, eps)
    b = joined(prec, R, R, eps, flags=E.EJOIN_FLAG_GATHER_RESCORE)
    same_bits(a, b)
    oi, oj, os_ = oracle.join(R, R, eps)
    compare(R, R, eps, a[0], a[1], a[2], oi, oj, os_)


def test_panels_cut_into_many_chunks():
    # eps = -1: every pair is a candidate, so each panel holds far more than one chunk of candidates
    R = np.random.default_rng(8).standard_normal((333, 48)).astype(np.float32)
    S = np.random.default_rng(9).standard_normal((5000, 48)).astype(np.float32)
    a = joined("bf16", R, S, -1.0)
    b = joined("bf16", R, S, -1.0, flags=E.EJOIN_FLAG_GATHER_RESCORE)
    same_bits(a, b)
    assert len(a[0]) == 333 * 5000
    want = oracle.sim_pairs(R, S, a[0].astype(np.uint32), a[1].astype(np.uint32))
    assert np.abs(a[2] - want).max() <= 1e-5


def test_panels_accurate_tier():
    # a wide FP64 band sends most candidates to the accurate tier, which both paths share
    d = 256
    rng = np.random.default_rng(10)
    centres = rng.standard_normal((20, d))
    R = clustered(11, 900, d, centres, 0.7)
    S = clustered(12, 1100, d, centres, 0.7)
    eps = 0.55
    a = joined("bf16", R, S, eps, fp64_band=0.2)
    b = joined("bf16", R, S, eps, fp64_band=0.2, flags=E.EJOIN_FLAG_GATHER_RESCORE)
    same_bits(a, b)
    assert a[3]["fp64_rescored"] > 1000
    oi, oj, os_ = oracle.join(R, S, eps)
    compare(R, S, eps, a[0], a[1], a[2], oi, oj, os_)
    # pairs the accurate tier decided carry its similarity: within FP32 rounding of the FP64 value
    near = np.abs(a[2] - eps) < 0.19
    assert near.sum() > 500
    want = oracle.sim_pairs(R, S, a[0][near].astype(np.uint32), a[1][near].astype(np.uint32))
    assert np.abs(a[2][near] - want).max() <= 1.2e-7


@pytest.mark.parametrize("d,pad", [(30, 0), (1030, 0), (64, 1)])
def test_shapes_outside_the_panel_kernel(d, pad):
    # d % 4 != 0, d > 1024, or rows not 16-byte aligned: the emission-order kernel runs instead
    rng = np.random.default_rng(d + pad)
    centres = rng.standard_normal((10, d))
    R = clustered(13, 400, d, centres, 0.5)
    S = clustered(14, 600, d, centres, 0.5)
    eps = 0.7
    if pad:
        # rows of ld = d + 1 floats: not 16-byte aligned
        Rp = np.zeros((len(R), d + 1), np.float32)
        Rp[:, :d] = R
        Rd = dev(Rp)[:, :d]
        with pkg.Ctx(device=0, prec="bf16") as ctx:
            res = pkg.ejoin_threshold(ctx, Rd, dev(S), eps)
        gi = res.i.cpu().numpy().view(np.uint32)
        gj = res.j.cpu().numpy().view(np.uint32)
        gs = res.sim.cpu().numpy()
    else:
        gi, gj, gs, _ = joined("bf16", R, S, eps)
    oi, oj, os_ = oracle.join(R, S, eps)
    assert len(oi) > 1000
    compare(R, S, eps, gi, gj, gs, oi, oj, os_)


def test_panels_count_only():
    d = 128
    rng = np.random.default_rng(15)
    centres = rng.standard_normal((25, d))
    R = clustered(16, 1200, d, centres, 0.6)
    S = clustered(17, 800, d, centres, 0.6)
    eps = 0.6
    full = joined("bf16", R, S, eps)
    with pkg.Ctx(device=0, prec="bf16", flags=E.EJOIN_FLAG_COUNT_ONLY) as ctx:
        pkg.ejoin_threshold(ctx, dev(R), dev(S), eps)
        st = pkg.ejoin_last_stats(ctx)
    assert st["pairs"] == len(full[0])


@pytest.mark.parametrize("d", [640, 768, 1024])
def test_sorted_clusters_take_the_s_major_path(d):
    # rows grouped by cluster (as the pruned join's reorder leaves them): a chunk's S rows then span a few
    # hundred positions and the chunk is processed S row by S row; same bits as the gather path
    rng = np.random.default_rng(d + 7)
    centres = rng.standard_normal((30, d))
    lab = np.sort(rng.integers(0, 30, 2400))
    centres = centres / np.linalg.norm(centres, axis=1, keepdims=True)
    X = (centres[lab] + rng.standard_normal((2400, d)) * (0.45 / np.sqrt(d))).astype(np.float32)
    X *= rng.uniform(0.5, 2.0, (2400, 1)).astype(np.float32)
    eps = 0.75
    for prec in ("bf16", "fp8"):
        a = joined(prec, X, X, eps)  # symmetric self-join (mirrored)
        b = joined(prec, X, X, eps, flags=E.EJOIN_FLAG_GATHER_RESCORE)
        same_bits(a, b)
        assert len(a[0]) > 100_000
    S = X[::-1].copy()  # a second relation, also grouped by cluster
    a = joined("bf16", X, S, eps)
    b = joined("bf16", X, S, eps, flags=E.EJOIN_FLAG_GATHER_RESCORE)
    same_bits(a, b)
    oi, oj, os_ = oracle.join(X, S, eps)
    compare(X, S, eps, a[0], a[1], a[2], oi, oj, os_)
