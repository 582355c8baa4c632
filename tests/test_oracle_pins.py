"""Pins for the FP64 oracle against facts that do not come from the oracle itself.

* closed forms derived by hand from Sec. III-A, Eq. (Cosine Similarity)
  (tests/golden/closed_form_cosines.txt);
* exact membership decided in rational arithmetic (Python ``fractions``) on
  the FP32 inputs, and exact similarities to 40 decimal digits;
* invariants implied by the algebra of Sec. III-C: eps <= -1 yields the full
  filtered cross product (Eq. theta-Join Generalization, Cartesian Product),
  eps > 1 yields nothing, self-join diagonal at 1, symmetry, monotonicity in
  eps, invariance to positive power-of-two scaling (Sec. IV-C: cosine equals
  the dot product of normalised rows), row-permutation equivariance (Sec. IV-C
  mapping back through offsets), selection pushdown commutes (Eq. E-Selection);
* planted near-duplicates that are matches by construction;
* mutation checks: each deliberately broken build of the oracle fails a pin.
"""
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
import ejoin_inputs as inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_cosines.txt")
getcontext().prec = 50


def _golden_cases():
    cases = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b, expr = [p.strip() for p in line.split(";")]
            a = np.array([float(t) for t in a.split()], dtype=np.float32)
            b = np.array([float(t) for t in b.split()], dtype=np.float32)
            val = eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt})
            cases.append((a, b, float(val)))
    return cases


# ----------------------------------------------------------------------------
# exact reference helpers (rational arithmetic on the exact FP32 input values)
# ----------------------------------------------------------------------------

def _exact_terms(a, b):
    fa = [Fraction(float(v)) for v in a]
    fb = [Fraction(float(v)) for v in b]
    dot = sum((x * y for x, y in zip(fa, fb)), Fraction(0))
    na = sum((x * x for x in fa), Fraction(0))
    nb = sum((y * y for y in fb), Fraction(0))
    return dot, na, nb


def exact_member(a, b, eps32) -> bool:
    """sim(a, b) >= eps decided exactly (zero row: sim = 0)."""
    dot, na, nb = _exact_terms(a, b)
    e = Fraction(float(eps32))
    if na == 0 or nb == 0:
        return 0 >= e
    P = na * nb
    if e <= 0:
        return dot >= 0 or dot * dot <= e * e * P
    return dot > 0 and dot * dot >= e * e * P


def exact_sim(a, b) -> Decimal:
    dot, na, nb = _exact_terms(a, b)
    if na == 0 or nb == 0:
        return Decimal(0)
    P = na * nb
    return (Decimal(dot.numerator) / Decimal(dot.denominator)) / (
        Decimal(P.numerator) / Decimal(P.denominator)).sqrt()


def _pairset(res):
    i, j, _ = res
    return set(zip(i.tolist(), j.tolist()))


def _rand_rel(rng, n, d, kind="float"):
    if kind == "int":
        x = rng.integers(-3, 4, size=(n, d)).astype(np.float32)
    else:
        x = rng.standard_normal((n, d)).astype(np.float32)
    return x


# ----------------------------------------------------------------------------
# pins
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("case", range(len(_golden_cases())))
def test_closed_forms(case):
    a, b, want = _golden_cases()[case]
    got = oracle.sim(a, b)
    assert abs(got - want) <= 4e-16, (a, b, got, want)
    assert abs(oracle.sim(b, a) - want) <= 4e-16


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("kind", ["float", "int"])
def test_exact_rational_membership(seed, kind):
    rng = np.random.default_rng(1000 + seed)
    R = _rand_rel(rng, 17, 6, kind)
    S = _rand_rel(rng, 13, 6, kind)
    R[3] = 0.0  # a zero row
    S[5] = -R[7]  # an antipodal pair
    S[6] = R[8] * 4  # a parallel pair
    for eps in (-1.0, -0.5, -0.01, 0.0, 0.3, 0.7, 0.95, 1.0):
        eps32 = np.float32(eps)
        got = _pairset(oracle.join(R, S, eps32))
        want, band = set(), set()
        for i in range(R.shape[0]):
            for j in range(S.shape[0]):
                if abs(exact_sim(R[i], S[j]) - Decimal(float(eps32))) < Decimal("1e-12"):
                    band.add((i, j))
                if exact_member(R[i], S[j], eps32):
                    want.add((i, j))
        assert (got ^ want) <= band, (eps, sorted(got ^ want))
    # similarities to FP64 accuracy
    i, j, s = oracle.join(R, S, -2.0)
    for a, b, v in zip(i, j, s):
        assert abs(Decimal(float(v)) - exact_sim(R[a], S[b])) < Decimal("1e-14")


def test_full_product_and_empty():
    rng = np.random.default_rng(7)
    R = _rand_rel(rng, 40, 9)
    S = np.concatenate([-R[:10], _rand_rel(rng, 25, 9)])  # 10 exactly antipodal pairs
    R[0] = 0.0
    attrR = rng.integers(0, 10, 40).astype(np.int32)
    attrS = rng.integers(0, 10, 35).astype(np.int32)
    selR, selS = oracle.Selection(attrR, "<", 6), oracle.Selection(attrS, ">=", 3)
    nR, nS = int((attrR < 6).sum()), int((attrS >= 3).sum())
    for eps in (-1.0, -1.5, -np.inf):
        assert len(oracle.join(R, S, eps, selR, selS)[0]) == nR * nS
        assert len(oracle.join(R, S, eps)[0]) == 40 * 35
    assert len(oracle.join(R, S, np.nextafter(np.float32(1), np.float32(2)))[0]) == 0
    assert len(oracle.join(R, S, 2.0)[0]) == 0
    # the antipodal pairs sit at -1 (to FP64 rounding) and are kept at eps = -1
    i, j, s = oracle.join(R[1:10], S[1:10], -1.0)
    anti = s[i == j]
    assert len(anti) == 9 and np.all(anti <= -1.0 + 1e-15)


def test_range_and_self_join_diagonal():
    rng = np.random.default_rng(11)
    X = _rand_rel(rng, 300, 37)
    X[5] = 0.0
    i, j, s = oracle.join(X, X, -1.0)
    assert s.min() >= -1.0 and s.max() <= 1.0
    diag = s[i == j]
    assert len(diag) == 300
    nz = np.arange(300) != 5
    assert np.all(diag[nz] >= 1.0 - 1e-15)
    assert diag[5] == 0.0
    # a zero row matches everything iff eps <= 0, and nothing above
    i, j, s = oracle.join(X, X, 0.0)
    assert np.sum(i == 5) == 300
    i, j, s = oracle.join(X, X, 1e-6)
    assert np.sum(i == 5) == 0
    # the diagonal of a self-join survives eps = 1 only via clamping to exactly 1
    i, j, s = oracle.join(X, X, 1.0)
    assert set(zip(i.tolist(), j.tolist())) <= {(k, k) for k in range(300)}


def test_symmetry_bitwise():
    rng = np.random.default_rng(12)
    X = _rand_rel(rng, 120, 33)
    i, j, s = oracle.join(X, X, 0.05)
    d = {(a, b): v for a, b, v in zip(i.tolist(), j.tolist(), s.tolist())}
    for (a, b), v in d.items():
        assert d[(b, a)] == v


def test_monotone_in_eps():
    rng = np.random.default_rng(13)
    R, S = _rand_rel(rng, 80, 7), _rand_rel(rng, 70, 7)
    prev = None
    for eps in (0.9, 0.6, 0.2, 0.0, -0.4, -1.0):
        cur = _pairset(oracle.join(R, S, eps))
        if prev is not None:
            assert prev <= cur
        prev = cur


def test_power_of_two_scaling_is_exact():
    rng = np.random.default_rng(14)
    R, S = _rand_rel(rng, 60, 24), _rand_rel(rng, 50, 24)
    base = oracle.join(R, S, 0.1)
    k = rng.integers(-6, 7, size=60).astype(np.float32)
    R2 = (R * np.exp2(k)[:, None]).astype(np.float32)
    S2 = (S * np.float32(2.0 ** 5)).astype(np.float32)
    got = oracle.join(R2, S2, 0.1)
    for a, b in zip(base, got):
        assert np.array_equal(a, b)


def test_row_permutation_equivariance():
    rng = np.random.default_rng(15)
    R, S = _rand_rel(rng, 64, 16), _rand_rel(rng, 48, 16)
    base = {(a, b): v for a, b, v in zip(*[x.tolist() for x in oracle.join(R, S, 0.2)])}
    pR, pS = rng.permutation(64), rng.permutation(48)
    i, j, s = oracle.join(R[pR], S[pS], 0.2)
    got = {(int(pR[a]), int(pS[b])): v for a, b, v in zip(i.tolist(), j.tolist(), s.tolist())}
    assert got == base


def test_basis_vectors_exact():
    d = 12
    E = np.eye(d, dtype=np.float32)
    X = np.concatenate([E, -E, 3 * E])
    i, j, s = oracle.join(X, X, -1.0)
    assert set(np.unique(s).tolist()) == {-1.0, 0.0, 1.0}
    # each e_k matches itself and 3 e_k at exactly 1, kept at eps = 1 (>=)
    i, j, s = oracle.join(X, X, 1.0)
    assert len(i) == 5 * d  # {E,3E} x {E,3E} on the same axis, and -E with -E
    assert np.all(s == 1.0)
    # orthogonal pairs sit exactly at 0 and are kept at eps = 0
    i, j, s = oracle.join(E, E, 0.0)
    assert len(i) == d * d


def test_selection_pushdown_commutes():
    rng = np.random.default_rng(16)
    R, S = _rand_rel(rng, 90, 10), _rand_rel(rng, 80, 10)
    aR = rng.integers(0, 1000, 90).astype(np.int32)
    aS = rng.integers(0, 1000, 80).astype(np.int32)
    full = oracle.join(R, S, 0.3)
    for opR, cR, opS, cS in (("<", 100, "<", 1000), ("<", 500, ">=", 300), ("==", aR[4], "!=", aS[2]),
                             (">", 900, "<=", 50)):
        sR, sS = oracle.Selection(aR, opR, cR), oracle.Selection(aS, opS, cS)
        got = _pairset(oracle.join(R, S, 0.3, sR, sS))
        keepR = {"<": aR < cR, ">": aR > cR, "==": aR == cR}[opR]
        keepS = {"<": aS < cS, ">=": aS >= cS, "!=": aS != cS, "<=": aS <= cS}[opS]
        want = {(a, b) for a, b in _pairset(full) if keepR[a] and keepS[b]}
        assert got == want
        assert oracle.count_selected(sR) == int(keepR.sum())


def test_sampled_rows_and_sim_pairs():
    rng = np.random.default_rng(17)
    R, S = _rand_rel(rng, 100, 20), _rand_rel(rng, 90, 20)
    full = oracle.join(R, S, 0.25)
    rows = [3, 17, 18, 60, 99]
    i, j, s = oracle.join(R, S, 0.25, rows=rows)
    mask = np.isin(full[0], rows)
    assert np.array_equal(i, full[0][mask]) and np.array_equal(j, full[1][mask])
    assert np.array_equal(s, full[2][mask])
    assert np.array_equal(oracle.sim_pairs(R, S, full[0], full[1]), full[2])


def test_output_sorted():
    rng = np.random.default_rng(18)
    R, S = _rand_rel(rng, 257, 5), _rand_rel(rng, 131, 5)
    i, j, _ = oracle.join(R, S, 0.5, threads=4)
    key = i.astype(np.int64) * 1000 + j
    assert np.all(np.diff(key) > 0)
    # thread count does not change the result
    for a, b in zip((i, j), oracle.join(R, S, 0.5, threads=1)[:2]):
        assert np.array_equal(a, b)


def test_planted_pairs_small():
    w = inputs.c1_planted(scale=0.25)
    i, j, s = oracle.join(w.R, w.S, w.eps)
    want = set(zip(w.extra["pi"].tolist(), w.extra["pj"].tolist()))
    assert set(zip(i.tolist(), j.tolist())) == want
    assert s.min() >= 0.95


@pytest.mark.slow
def test_planted_pairs_c1_full():
    """4096 x 4096 x 128 at eps 0.9: exactly the 64 planted pairs (chance matches of
    i.i.d. Gaussian rows at cos >= 0.9 in 128-d are ~10 sigma events)."""
    w = inputs.c1_planted()
    i, j, s = oracle.join(w.R, w.S, w.eps)
    want = set(zip(w.extra["pi"].tolist(), w.extra["pj"].tolist()))
    assert set(zip(i.tolist(), j.tolist())) == want
    assert len(i) == 64


# ----------------------------------------------------------------------------
# mutation checks: a plausible mistake anywhere in the oracle fails a pin
# ----------------------------------------------------------------------------

def _pins_pass(mutant: int) -> bool:
    try:
        for a, b, want in _golden_cases():
            if abs(oracle.sim(a, b, mutant=mutant) - want) > 4e-16:
                return False
        d = 12
        E = np.eye(d, dtype=np.float32)
        X = np.concatenate([E, -E])
        if len(oracle.join(X, X, -1.0, mutant=mutant)[0]) != (2 * d) ** 2:
            return False
        if len(oracle.join(E, E, 1.0, mutant=mutant)[0]) != d:
            return False
        rng = np.random.default_rng(11)
        Y = _rand_rel(rng, 300, 37)
        s = oracle.join(Y, Y, -1.0, mutant=mutant)[2]
        if s.max() > 1.0 or s.min() < -1.0:
            return False
        return True
    except Exception:
        return False


def _top1_pins_pass(mutant: int) -> bool:
    """Top-1: exact argmax (rational arithmetic) on small integer rows, with ties to the smaller j."""
    try:
        rng = np.random.default_rng(31)
        for trial in range(4):
            R = _rand_rel(rng, 9, 4, "int")
            S = _rand_rel(rng, 13, 4, "int")
            S[7] = S[2]  # an exact tie: j = 2 must win over j = 7 wherever S[2] is the best
            oi, oj, os_ = oracle.top1(R, S, mutant=mutant)
            for i, j, sv in zip(oi.tolist(), oj.tolist(), os_.tolist()):
                sims = [exact_sim(R[i], S[k]) for k in range(len(S))]
                best = max(sims)
                want = min(k for k, v in enumerate(sims) if v == best)
                if j != want or abs(Decimal(sv) - best) > Decimal("1e-15"):
                    return False
        return True
    except Exception:
        return False


def _topk_pins_pass(mutant: int) -> bool:
    """Top-k: each row's list holds min(k, |S|) distinct rows whose exact (rational) similarities are the
    k largest, in descending order; a row left out that ties exactly with a listed one has the larger j."""
    try:
        rng = np.random.default_rng(37)
        for trial in range(4):
            R = _rand_rel(rng, 7, 4, "int")
            S = _rand_rel(rng, 15, 4, "int")
            S[9] = S[3]  # exact duplicates: equal similarities in any arithmetic
            S[12] = S[3]
            S[14] = S[5]
            for k in (1, 2, 3, 5, 15, 17):
                oi, oj, os_ = oracle.topk(R, S, k, mutant=mutant)
                kk = min(k, len(S))
                if list(oi) != [i for i in range(len(R)) for _ in range(kk)]:
                    return False
                for i in range(len(R)):
                    js = oj[i * kk:(i + 1) * kk].tolist()
                    ss = os_[i * kk:(i + 1) * kk].tolist()
                    ex = [exact_sim(R[i], S[j]) for j in range(len(S))]
                    top = sorted(ex, reverse=True)[:kk]
                    if len(set(js)) != kk:
                        return False
                    for t, (j, v) in enumerate(zip(js, ss)):
                        if abs(Decimal(v) - ex[j]) > Decimal("1e-15") or abs(ex[j] - top[t]) > Decimal("1e-15"):
                            return False
                        if t and (v > ss[t - 1] or (v == ss[t - 1] and j < js[t - 1])):
                            return False
                    for j in set(range(len(S))) - set(js):
                        if any(np.array_equal(S[j], S[jj]) and jj > j for jj in js):
                            return False
        return True
    except Exception:
        return False


def test_oracle_passes_pins():
    assert _pins_pass(0)
    assert _top1_pins_pass(0)
    assert _topk_pins_pass(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7, 8])
def test_mutants_are_caught(mutant):
    assert not (_pins_pass(mutant) and _top1_pins_pass(mutant) and _topk_pins_pass(mutant))


def test_topk_agrees_with_top1_and_the_threshold_join():
    # k = 1 is the top-1 condition; each row's k records are the threshold join at eps just below its
    # k-th similarity, whenever the k-th and (k+1)-th similarities differ (Sec. VI-E: the top-k and range
    # conditions on the same product)
    rng = np.random.default_rng(47)
    R, S = _rand_rel(rng, 30, 19), _rand_rel(rng, 70, 19)
    a, b = oracle.topk(R, S, 1), oracle.top1(R, S)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    k = 6
    oi, oj, os_ = oracle.topk(R, S, k)
    assert len(oi) == 30 * k
    for i in range(30):
        sims = os_[i * k:(i + 1) * k]
        eps = float(np.nextafter(np.float32(sims[-1]), np.float32(-2)))
        ji, jj, js = oracle.join(R[i:i + 1], S, eps)
        assert set(oj[i * k:(i + 1) * k].tolist()) <= set(jj.tolist())
        assert len(jj) >= k and np.all(np.diff(sims) <= 0)


def test_topk_selection_and_short_relations():
    rng = np.random.default_rng(53)
    R, S = _rand_rel(rng, 25, 11), _rand_rel(rng, 40, 11)
    aR, aS = rng.integers(0, 10, 25).astype(np.int32), rng.integers(0, 10, 40).astype(np.int32)
    oi, oj, os_ = oracle.topk(R, S, 4, oracle.Selection(aR, ">=", 5), oracle.Selection(aS, "<", 2))
    keepS = np.nonzero(aS < 2)[0]
    kk = min(4, len(keepS))
    fi, fj, fs = oracle.topk(R, S[keepS], 4)
    want_rows = np.nonzero(aR >= 5)[0]
    assert np.array_equal(oi, np.repeat(want_rows, kk).astype(np.uint32))
    sel = np.isin(fi, want_rows)
    assert np.array_equal(oj, keepS[fj[sel]]) and np.array_equal(os_, fs[sel])
    # k larger than S: every kept S row, sorted
    oi, oj, os_ = oracle.topk(R[:3], S[:5], 9)
    assert len(oi) == 15 and all(sorted(oj[t * 5:(t + 1) * 5].tolist()) == list(range(5)) for t in range(3))


def test_top1_is_the_best_pair_of_the_threshold_join():
    # for each R row, the threshold join at eps just below the top-1 similarity holds the top-1 pair
    # and no pair of larger similarity (Sec. VI-E: the top-k and range conditions on the same product)
    rng = np.random.default_rng(41)
    R, S = _rand_rel(rng, 40, 23), _rand_rel(rng, 60, 23)
    oi, oj, os_ = oracle.top1(R, S)
    assert list(oi) == list(range(40))
    for i, j, sv in zip(oi.tolist(), oj.tolist(), os_.tolist()):
        eps = float(np.nextafter(np.float32(sv), np.float32(-2)))
        ji, jj, js = oracle.join(R[i:i + 1], S, eps)
        assert j in set(jj.tolist()) and js.max() <= sv


def test_top1_selection_and_permutation():
    rng = np.random.default_rng(43)
    R, S = _rand_rel(rng, 30, 17), _rand_rel(rng, 50, 17)
    aR, aS = rng.integers(0, 10, 30).astype(np.int32), rng.integers(0, 10, 50).astype(np.int32)
    oi, oj, os_ = oracle.top1(R, S, oracle.Selection(aR, "<", 6), oracle.Selection(aS, ">=", 3))
    keepS = np.nonzero(aS >= 3)[0]
    fi, fj, fs = oracle.top1(R, S[keepS])
    want = {i: (keepS[j], v) for i, j, v in zip(fi.tolist(), fj.tolist(), fs.tolist()) if aR[i] < 6}
    assert set(oi.tolist()) == set(want)
    for i, j, v in zip(oi.tolist(), oj.tolist(), os_.tolist()):
        assert j == want[i][0] and v == want[i][1]
    perm = rng.permutation(50)
    pi, pj, ps = oracle.top1(R, S[perm])
    base = oracle.top1(R, S)
    assert np.array_equal(perm[pj], base[1]) and np.array_equal(ps, base[2])
