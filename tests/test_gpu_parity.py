"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes span several 128 x 256 tiles with ragged tails; every precision runs the
same cases.  The comparison rule is in parity_util: identical pair sets
outside |sim - eps| < 1e-5, similarities within 1e-5.
"""
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

PRECS = ["f32", "bf16", "tf32", "fp8"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(prec, R, S, eps, selR=None, selS=None, capacity=None, **kw):
    with pkg.Ctx(device=0, prec=prec, **kw) as ctx:
        res = pkg.ejoin_threshold(ctx, dev(R), dev(S), eps, selR, selS, capacity=capacity)
        torch.cuda.synchronize()
        stats = pkg.ejoin_last_stats(ctx)
        return (res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32),
                res.sim.cpu().numpy(), stats)


def gauss(seed, n, d):
    return np.random.default_rng(seed).standard_normal((n, d)).astype(np.float32)


@pytest.mark.parametrize("prec", PRECS)
def test_planted_pairs(prec):
    w = inputs.c1_planted(scale=0.25)
    gi, gj, gs, st = run(prec, w.R, w.S, w.eps)
    oi, oj, os_ = oracle.join(w.R, w.S, w.eps)
    assert len(oi) == 64
    compare(w.R, w.S, w.eps, gi, gj, gs, oi, oj, os_)
    assert set(zip(gi.tolist(), gj.tolist())) == set(zip(w.extra["pi"].tolist(), w.extra["pj"].tolist()))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(300, 700, 37), (129, 257, 128), (1000, 513, 300), (37, 2000, 64)])
def test_random_ragged(prec, shape):
    nR, nS, d = shape
    R, S = gauss(1, nR, d), gauss(2, nS, d)
    eps = 0.25 if d < 64 else 0.12
    gi, gj, gs, st = run(prec, R, S, eps)
    oi, oj, os_ = oracle.join(R, S, eps)
    assert len(oi) > 50
    compare(R, S, eps, gi, gj, gs, oi, oj, os_)


@pytest.mark.parametrize("prec", PRECS)
def test_selection_both_sides(prec):
    rng = np.random.default_rng(3)
    R, S = gauss(4, 3000, 100), gauss(5, 1500, 100)
    aR = rng.integers(0, 1000, 3000).astype(np.int32)
    aS = rng.integers(0, 1000, 1500).astype(np.int32)
    bits = rng.integers(0, 2**32, (1500 + 31) // 32, dtype=np.uint32)
    eps = 0.2
    selR = pkg.Sel(dev(aR), "<", 300)
    selS = pkg.Sel(dev(aS), ">=", 500, bits=dev(bits.view(np.int32)))
    gi, gj, gs, st = run(prec, R, S, eps, selR, selS)
    keepS = (aS >= 500) & (((bits[np.arange(1500) // 32] >> (np.arange(1500) % 32)) & 1) == 1)
    # the oracle evaluates attr predicates itself; the bitmask is applied as a second predicate column
    mask_attr = np.where(keepS, 1, 0).astype(np.int32)
    oi, oj, os_ = oracle.join(R, S, eps, oracle.Selection(aR, "<", 300), oracle.Selection(mask_attr, "==", 1))
    compare(R, S, eps, gi, gj, gs, oi, oj, os_)
    assert st["n_sel_r"] == int((aR < 300).sum())
    assert st["n_sel_s"] == int(keepS.sum())


@pytest.mark.parametrize("prec", PRECS)
def test_full_product_and_empty(prec):
    R, S = gauss(6, 200, 48), gauss(7, 333, 48)
    R[:10] = -S[:10]  # exactly antipodal rows
    gi, gj, gs, st = run(prec, R, S, -1.0)
    assert len(gi) == 200 * 333
    assert len(set(zip(gi.tolist(), gj.tolist()))) == 200 * 333
    gi, gj, gs, st = run(prec, R, S, float(np.nextafter(np.float32(1), np.float32(2))))
    assert len(gi) == 0


@pytest.mark.parametrize("prec", PRECS)
def test_self_join_diagonal_and_symmetry(prec):
    X = gauss(8, 700, 96)
    X[13] = 0.0  # zero row: similarity 0 with everything
    eps = 0.3
    gi, gj, gs, st = run(prec, X, X, eps)
    oi, oj, os_ = oracle.join(X, X, eps)
    compare(X, X, eps, gi, gj, gs, oi, oj, os_)
    d = dict(zip(zip(gi.tolist(), gj.tolist()), gs.tolist()))
    for k in range(700):
        if k != 13:
            assert abs(d[(k, k)] - 1.0) <= 1e-5
    assert not any(a == 13 or b == 13 for a, b in d)
    for (a, b) in d:
        assert (b, a) in d


@pytest.mark.parametrize("prec", PRECS)
def test_scaled_rows_and_padding_dims(prec):
    # non-unit rows with large and tiny magnitudes; d not a multiple of any tile
    rng = np.random.default_rng(9)
    R = gauss(10, 400, 301) * np.exp2(rng.integers(-40, 40, 400)).astype(np.float32)[:, None]
    S = gauss(11, 300, 301) * np.float32(1e-20)
    S[:40] = R[:40] * np.float32(3.0)
    eps = 0.15
    gi, gj, gs, st = run(prec, R, S, eps)
    oi, oj, os_ = oracle.join(R, S, eps)
    compare(R, S, eps, gi, gj, gs, oi, oj, os_)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_candidate_buffer_regrowth(prec):
    R, S = gauss(12, 500, 64), gauss(13, 400, 64)
    eps = -0.05  # about half of all pairs
    # the candidate buffer exists on the two-kernel path (the fused kernel has no candidate buffer)
    gi, gj, gs, st = run(prec, R, S, eps, capacity=1 << 20, capacity_hint=64)
    assert st["contract_retries"] >= 1
    oi, oj, os_ = oracle.join(R, S, eps)
    compare(R, S, eps, gi, gj, gs, oi, oj, os_)


def test_empty_inputs_and_empty_selection():
    R, S = gauss(14, 100, 32), gauss(15, 90, 32)
    for prec in ("f32", "bf16"):
        gi, gj, gs, st = run(prec, R[:0], S, 0.1)
        assert len(gi) == 0
        gi, gj, gs, st = run(prec, R, S[:0], 0.1)
        assert len(gi) == 0
        attr = np.zeros(100, dtype=np.int32)
        gi, gj, gs, st = run(prec, R, S, -1.0, pkg.Sel(dev(attr), ">", 5))
        assert len(gi) == 0 and st["n_sel_r"] == 0


def test_nonfinite_input_is_reported():
    R, S = gauss(16, 50, 32), gauss(17, 60, 32)
    R[7, 3] = np.nan
    with pytest.raises(pkg.EJoinError) as e:
        run("bf16", R, S, 0.5)
    assert e.value.status == 4
    R[7, 3] = np.inf
    with pytest.raises(pkg.EJoinError) as e:
        run("f32", R, S, 0.5)
    assert e.value.status == 4


def test_overflow_status_and_count():
    import ctypes
    from paper_2312_01476_gb300 import ejoin as E
    R, S = gauss(18, 300, 40), gauss(19, 200, 40)
    lib = E.load_library()
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        out_t = torch.empty((10, 3), dtype=torch.int32, device="cuda")
        cnt_t = torch.zeros(1, dtype=torch.int64, device="cuda")
        out = E.ejoin_pairs(ctypes.c_void_p(out_t.data_ptr()), 10, ctypes.c_void_p(cnt_t.data_ptr()), 0)
        Rd, Sd = dev(R), dev(S)
        st = lib.ejoin_threshold(ctx.handle, E._dev_rel(Rd), E._dev_rel(Sd), ctypes.c_float(-1.0), None, None,
                                 ctypes.byref(out))
        assert st == E.EJOIN_EOVERFLOW
        assert out.count == 300 * 200 and int(cnt_t.item()) == 300 * 200
        # library-allocated buffer
        out2 = E.ejoin_pairs(None, 0, None, 0)
        st = lib.ejoin_threshold(ctx.handle, E._dev_rel(Rd), E._dev_rel(Sd), ctypes.c_float(0.2), None, None,
                                 ctypes.byref(out2))
        assert st == 0 and out2.d_pairs and out2.capacity >= out2.count
        assert lib.ejoin_pairs_free(ctx.handle, ctypes.byref(out2)) == 0


def test_invalid_arguments():
    import ctypes
    from paper_2312_01476_gb300 import ejoin as E
    lib = E.load_library()
    R, S = dev(gauss(20, 10, 8)), dev(gauss(21, 10, 9))
    with pkg.Ctx(device=0, prec="f32") as ctx:
        out = E.ejoin_pairs(None, 0, None, 0)
        assert lib.ejoin_threshold(ctx.handle, E._dev_rel(R), E._dev_rel(S), ctypes.c_float(0.1), None, None,
                                   ctypes.byref(out)) == E.EJOIN_EINVAL
        assert lib.ejoin_threshold(ctx.handle, E._dev_rel(R), E._dev_rel(R), ctypes.c_float(float("nan")), None,
                                   None, ctypes.byref(out)) == E.EJOIN_EINVAL


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_host_api_matches_device_api(prec):
    w = inputs.c2_clustered_selection(nR=20000, nS=3000, d=300, n_clusters=50, threads=4)
    with pkg.Ctx(device=0, prec=prec) as ctx:
        pairs, n = pkg.ejoin_threshold_host(ctx, w.R, w.S, w.eps, pkg.Sel(w.attrR, "<", w.cR))
    oi, oj, os_ = oracle.join(w.R, w.S, w.eps, oracle.Selection(w.attrR, "<", w.cR))
    assert n == len(pairs) and n > 1000
    compare(w.R, w.S, w.eps, pairs["i"], pairs["j"], pairs["sim"], oi, oj, os_)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "tf32", "f32"])
def test_host_api_reads_pinned_inputs_in_place(prec):
    # pinned host inputs: the predicates and the kept rows are read in place (only they cross the link);
    # the result equals the whole-copy route's and the oracle's
    w = inputs.c2_clustered_selection(nR=20000, nS=3000, d=300, n_clusters=50, threads=4)
    aS = np.random.default_rng(5).integers(0, 10, 3000).astype(np.int32)

    def pin(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    Rp, Sp, Ap, aSp = pin(w.R), pin(w.S), pin(w.attrR), pin(aS)
    outp = torch.empty(12 * 400000, dtype=torch.uint8).pin_memory().numpy().view(pkg.PAIR_DTYPE)
    with pkg.Ctx(device=0, prec=prec) as ctx:
        # a pinned result buffer too: the re-score writes the pairs into it directly
        pairs, n = pkg.ejoin_threshold_host(ctx, Rp, Sp, w.eps, pkg.Sel(Ap, "<", w.cR), pkg.Sel(aSp, "<", 7),
                                            out=outp)
        st = pkg.ejoin_last_stats(ctx)
    n_r, n_s = int((w.attrR < w.cR).sum()), int((aS < 7).sum())
    assert st["host_in_place"] == 1
    assert st["h2d_bytes"] == (n_r + n_s) * 300 * 4 + (20000 + 3000) * 4
    oi, oj, os_ = oracle.join(w.R, w.S, w.eps, oracle.Selection(w.attrR, "<", w.cR), oracle.Selection(aS, "<", 7))
    assert n > 100
    compare(w.R, w.S, w.eps, pairs["i"], pairs["j"], pairs["sim"], oi, oj, os_)
    with pkg.Ctx(device=0, prec=prec, flags=pkg.EJOIN_FLAG_HOST_COPY) as ctx:
        pairs2, n2 = pkg.ejoin_threshold_host(ctx, Rp, Sp, w.eps, pkg.Sel(Ap, "<", w.cR), pkg.Sel(aSp, "<", 7))
        st2 = pkg.ejoin_last_stats(ctx)
    assert st2["host_in_place"] == 0 and st2["h2d_bytes"] == (20000 + 3000) * 300 * 4 + (20000 + 3000) * 4
    a = np.sort(pairs[["i", "j", "sim"]], order=["i", "j"])
    b = np.sort(pairs2[["i", "j", "sim"]], order=["i", "j"])
    assert np.array_equal(a, b)


def test_host_api_pinned_self_join():
    # a pinned self-join: one operand read in place, the symmetric evaluation mirrored in the re-score
    X = gauss(41, 3000, 96)
    X[1500:1600] = X[:100] + 0.05 * gauss(42, 100, 96)
    Xp = torch.from_numpy(X).pin_memory().numpy()
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        pairs, n = pkg.ejoin_threshold_host(ctx, Xp, Xp, 0.6)
        st = pkg.ejoin_last_stats(ctx)
    assert st["host_in_place"] == 1 and st["h2d_bytes"] == 3000 * 96 * 4
    oi, oj, os_ = oracle.join(X, X, 0.6)
    compare(X, X, 0.6, pairs["i"], pairs["j"], pairs["sim"], oi, oj, os_)


def test_normalize_entry_point():
    X = gauss(22, 1000, 300)
    attr = np.arange(1000, dtype=np.int32) % 7
    Xd = dev(X)
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        for prec in ("f32", "bf16", "fp8"):
            out, inv, scale, ids, n_sel = pkg.ejoin_normalize(ctx, Xd, prec, pkg.Sel(dev(attr), "==", 3))
            torch.cuda.synchronize()
            n = int(n_sel.item())
            assert n == oracle.count_selected(oracle.Selection(attr, "==", 3))
            assert np.array_equal(ids[:n].cpu().numpy(), np.nonzero(attr == 3)[0])
            rows = out[:n].float().cpu().numpy().astype(np.float64)
            if prec == "fp8":
                rows = out[:n].cpu().view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
                rows *= scale[:n].cpu().numpy()[:, None]
            norms = np.linalg.norm(rows, axis=1)
            tol = {"f32": 1e-6, "bf16": 1e-2, "fp8": 0.13}[prec]
            assert np.all(np.abs(norms - 1) <= tol), (prec, np.abs(norms - 1).max())
            assert np.all(rows[:, 300:] == 0)
            exact = [1.0 / oracle.norm(X[r]) for r in np.nonzero(attr == 3)[0]]
            assert np.allclose(inv[:n].cpu().numpy(), exact, rtol=1e-6)


@pytest.mark.parametrize("d", [4, 200, 384, 512, 700, 768, 1024, 1030])
@pytest.mark.parametrize("prec", ["bf16", "f32"])
def test_dims_cover_every_rescore_variant(prec, d):
    # d picks the re-score kernel variant (row gathers of 1..8 float4 per lane, or the generic loop)
    R, S = gauss(30 + d, 260, d), gauss(31 + d, 300, d)
    S[:50] = R[:50] + np.float32(0.3) * gauss(32 + d, 50, d)
    eps = 0.5 if d > 8 else 0.7
    gi, gj, gs, st = run(prec, R, S, eps)
    oi, oj, os_ = oracle.join(R, S, eps)
    assert len(oi) >= 40
    compare(R, S, eps, gi, gj, gs, oi, oj, os_)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "tf32"])
def test_fused_and_two_kernel_paths_agree(prec):
    # eps in the middle of the intra-cluster similarities (0.913 +- 0.005): band-heavy, FP64 tier busy
    w = inputs.c2_clustered_selection(nR=60000, nS=9000, d=300, n_clusters=40, threads=4, eps=0.912)
    selR = pkg.Sel(dev(w.attrR), "<", w.cR)
    gi, gj, gs, st = run(prec, w.R, w.S, w.eps, selR, capacity=1 << 22, fp64_band=0.02, flags=pkg.EJOIN_FLAG_FUSED)
    assert st["fused"] == 1 and st["fp64_rescored"] > 0
    ui, uj, us, su = run(prec, w.R, w.S, w.eps, selR, capacity=1 << 22, fp64_band=0.02)
    assert su["fused"] == 0
    a = dict(zip(zip(gi.tolist(), gj.tolist()), gs.tolist()))
    b = dict(zip(zip(ui.tolist(), uj.tolist()), us.tolist()))
    assert set(a) == set(b) and len(a) > 10000
    assert max(abs(a[k] - b[k]) for k in a) == 0.0  # same arithmetic per candidate
    rows = np.sort(np.random.default_rng(1).choice(np.nonzero(w.attrR < w.cR)[0], 40, replace=False))
    oi, oj, os_ = oracle.join(w.R, w.S, w.eps, oracle.Selection(w.attrR, "<", w.cR), rows=rows)
    compare(w.R, w.S, w.eps, gi, gj, gs, oi, oj, os_, rows=rows)
    assert st["candidates"] == su["candidates"]


def test_fused_path_counts_beyond_the_result_buffer():
    R, S = gauss(40, 700, 64), gauss(41, 500, 64)
    with pkg.Ctx(device=0, prec="bf16", flags=pkg.EJOIN_FLAG_FUSED) as ctx:
        res = pkg.ejoin_threshold(ctx, dev(R), dev(S), -1.0, capacity=1000)  # overflow, then retry
        assert res.count == 700 * 500
        assert pkg.ejoin_last_stats(ctx)["fused"] == 1


@pytest.mark.parametrize("shape", [(129, 257, 128), (1000, 513, 300), (300, 700, 40)])
def test_fused_path_matches_oracle_dense(shape):
    # candidate-dense joins drive the fused kernel's shared-memory ring through many laps
    nR, nS, d = shape
    R, S = gauss(50 + d, nR, d), gauss(51 + d, nS, d)
    for prec in ("bf16", "fp8"):
        # eps = 0.02: about 45 % of the Gaussian pairs are candidates at every d here
        gi, gj, gs, st = run(prec, R, S, 0.02, capacity=1 << 22, flags=pkg.EJOIN_FLAG_FUSED)
        assert st["fused"] == 1 and st["candidates"] > 0.3 * nR * nS
        oi, oj, os_ = oracle.join(R, S, 0.02)
        compare(R, S, 0.02, gi, gj, gs, oi, oj, os_)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "tf32"])
@pytest.mark.parametrize("n", [300, 256, 513, 1500])
def test_symmetric_self_join_equals_full_square(prec, n):
    # the upper-triangle evaluation (default for tensor-core self-joins) returns the same set as the
    # full square, every off-diagonal pair in both orders with one similarity, and matches the oracle
    X = gauss(60 + n, n, 96)
    X[n // 2:] = X[: n - n // 2] + np.float32(0.4) * gauss(61 + n, n - n // 2, 96)
    eps = 0.3
    Xd = dev(X)  # one tensor for both sides: a self-join is recognised by identical relations

    def run_self(flags=0):
        with pkg.Ctx(device=0, prec=prec, flags=flags) as ctx:
            res = pkg.ejoin_threshold(ctx, Xd, Xd, eps)
            return (res.i.cpu().numpy().view(np.uint32), res.j.cpu().numpy().view(np.uint32),
                    res.sim.cpu().numpy(), pkg.ejoin_last_stats(ctx))

    gi, gj, gs, st = run_self()
    fi, fj, fs, sf = run_self(pkg.EJOIN_FLAG_NO_SYMMETRY)
    assert st["candidates"] < sf["candidates"]
    a = dict(zip(zip(gi.tolist(), gj.tolist()), gs.tolist()))
    b = dict(zip(zip(fi.tolist(), fj.tolist()), fs.tolist()))
    assert len(a) == len(gi) and set(a) == set(b)
    assert all(a[(i, j)] == a[(j, i)] for (i, j) in a)
    assert all((i, i) in a for i in range(n))
    oi, oj, os_ = oracle.join(X, X, eps)
    compare(X, X, eps, gi, gj, gs, oi, oj, os_)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "f32"])
@pytest.mark.parametrize("d", [768, 299])
def test_accurate_tier_matches_fp64(prec, d):
    # fp64_band = 2 sends every candidate through the accurate tier (compensated dot products finished
    # in FP64): its similarities then agree with the FP64 oracle to FP32 rounding of the result
    # (|err| <= 2^-24 for |sim| <= 1) plus the tier's own bound (< 3e-9 at d = 768); d = 299 takes the
    # scalar-load variant of the tier
    R, S = gauss(70, 700, d), gauss(71, 900, d)
    S[:300] = R[:300] + np.float32(0.35) * gauss(72, 300, d)
    R[:5] *= np.float32(1e-3)  # rows far from unit length
    S[5:10] *= np.float32(1e3)
    eps = 0.2
    gi, gj, gs, st = run(prec, R, S, eps, fp64_band=2.0)
    assert st["fp64_rescored"] == st["candidates"] > 0
    oi, oj, os_ = oracle.join(R, S, eps)
    compare(R, S, eps, gi, gj, gs, oi, oj, os_, band=1e-7, tol=1.2e-7)


@pytest.mark.parametrize("prec", ["bf16", "f32"])
def test_library_allocated_result_self_join(prec):
    # out->d_pairs == NULL: the library sizes the buffer itself; a symmetric self-join writes every
    # off-diagonal pair twice, so the buffer must hold twice its candidates
    import ctypes
    from paper_2312_01476_gb300 import ejoin as E
    X = gauss(31, 900, 64)
    X[450:] = X[:450] + np.float32(0.2) * gauss(32, 450, 64)
    eps = 0.5
    lib = E.load_library()
    with pkg.Ctx(device=0, prec=prec) as ctx:
        Xd = dev(X)
        out = E.ejoin_pairs(None, 0, None, 0)
        st = lib.ejoin_threshold(ctx.handle, E._dev_rel(Xd), E._dev_rel(Xd), ctypes.c_float(eps), None, None,
                                 ctypes.byref(out))
        assert st == 0, pkg.ejoin_strerror(st)
        n = int(out.count)
        assert out.d_pairs and out.capacity >= n
        assert lib.ejoin_pairs_free(ctx.handle, ctypes.byref(out)) == 0
        want = pkg.ejoin_threshold(ctx, Xd, Xd, eps)  # the binding's caller-owned buffer (checked elsewhere)
    assert n == want.count and n > 2 * len(X)
