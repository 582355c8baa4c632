"""Batched E-joins (one persistent launch over a job table, CUDA-graph replay,
autotuned raster): every job's pairs equal the FP64 oracle's for that job
under the parity rule of parity_util."""
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


def make_jobs(seed, sizes, d, eps_lo=0.3, eps_hi=0.6, planted=True):
    rng = np.random.default_rng(seed)
    jobs_np = []
    for k, (nR, nS) in enumerate(sizes):
        R = rng.standard_normal((nR, d)).astype(np.float32)
        S = rng.standard_normal((nS, d)).astype(np.float32)
        if planted and nR and nS:
            m = min(nR, nS, 20)
            S[:m] = R[:m] + np.float32(0.4) * rng.standard_normal((m, d)).astype(np.float32)
        eps = float(rng.uniform(eps_lo, eps_hi))
        jobs_np.append((R, S, eps))
    return jobs_np


def check_batch(jobs_np, job, gi, gj, gs):
    for k, (R, S, eps) in enumerate(jobs_np):
        sel = job == k
        oi, oj, os_ = oracle.join(R, S, eps)
        compare(R, S, eps, gi[sel], gj[sel], gs[sel], oi, oj, os_)


def to_dev(jobs_np):
    return [(torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda(), eps) for R, S, eps in jobs_np]


SIZES = [(300, 700), (0, 50), (40, 0), (1, 1), (129, 257), (1000, 513), (37, 2000), (256, 256), (5, 900),
         (777, 31)]


@pytest.mark.parametrize("prec", ["bf16", "fp8", "tf32"])
def test_batch_matches_oracle_per_job(prec):
    jobs_np = make_jobs(1, SIZES, 96)
    with pkg.Ctx(device=0, prec=prec) as ctx:
        job, gi, gj, gs = pkg.ejoin_batch(ctx, to_dev(jobs_np), graph=True)
    assert len(job) > 100
    check_batch(jobs_np, job, gi.view(np.uint32), gj.view(np.uint32), gs)


def test_batch_graph_replay_is_stable_and_autotuned():
    jobs_np = make_jobs(2, SIZES[::-1] + [(2000, 1500)], 128, 0.2, 0.5)
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        b = pkg.Batch(ctx, to_dev(jobs_np), graph=True, autotune=True)
        info = b.info()
        assert info["graph"] == 1 and info["group_m"] in (4, 8, 16, 32, 64, 128)
        sets = []
        for _ in range(3):
            b.run()
        n = b.wait()
        for _ in range(2):
            b.run()
            n2 = b.wait()
            assert n2 == n
            job, gi, gj, gs = (x.cpu().numpy() for x in b.result(n2))
            sets.append(set(zip(job.tolist(), gi.tolist(), gj.tolist())))
        assert sets[0] == sets[1]
        check_batch(jobs_np, job, gi.view(np.uint32), gj.view(np.uint32), gs)
        b.close()


def test_batch_unaligned_rows_use_the_generic_rescore():
    rng = np.random.default_rng(3)
    jobs_np = []
    jobs_dev = []
    for nR, nS in [(200, 300), (150, 90)]:
        Rw = rng.standard_normal((nR, 67)).astype(np.float32)
        Sw = rng.standard_normal((nS, 67)).astype(np.float32)
        # d = 66 with ld = 67: rows are not 16-byte aligned
        jobs_np.append((np.ascontiguousarray(Rw[:, :66]), np.ascontiguousarray(Sw[:, :66]), 0.3))
        jobs_dev.append((torch.from_numpy(Rw).cuda()[:, :66], torch.from_numpy(Sw).cuda()[:, :66], 0.3))
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        job, gi, gj, gs = pkg.ejoin_batch(ctx, jobs_dev, graph=False)
    check_batch(jobs_np, job, gi.view(np.uint32), gj.view(np.uint32), gs)


def test_batch_clustered_lognormal_small():
    # the shape of the batched workload at a scale the oracle finishes in seconds
    rng = np.random.default_rng(inputs.seed_for(4))
    d = 384
    centres = inputs.sphere_centres(50, d, inputs.seed_for(4))
    jobs_np = []
    for k in range(16):
        nR, nS = np.clip(np.round(np.exp(rng.normal(np.log(300), 1.0, 2))), 20, 3000).astype(int)
        R = inputs.clustered(int(nR), d, centres, 0.3, inputs.seed_for(4) * 1000 + 2 * k, threads=1)
        S = inputs.clustered(int(nS), d, centres, 0.3, inputs.seed_for(4) * 1000 + 2 * k + 1, threads=1)
        jobs_np.append((R, S, float(rng.uniform(0.8, 0.95))))
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        job, gi, gj, gs = pkg.ejoin_batch(ctx, to_dev(jobs_np), graph=True)
    assert len(job) > 1000
    check_batch(jobs_np, job, gi.view(np.uint32), gj.view(np.uint32), gs)


def records(ctx_kw, jobs_dev, flags=0):
    with pkg.Ctx(device=0, flags=flags, **ctx_kw) as ctx:
        job, gi, gj, gs = pkg.ejoin_batch(ctx, jobs_dev, graph=True)
        st = pkg.ejoin_last_stats(ctx)
    key = (job.astype(np.int64) << 42) | (gi.view(np.uint32).astype(np.int64) << 21) | gj.view(np.uint32)
    o = np.argsort(key)
    return key[o], gs[o].view(np.uint32), st


# row widths of every streaming instantiation (V = 1, 2, 3, 4, 6, 8 float4 per lane), with rows that fill
# the lanes exactly (128, 256, 384, 512, 768, 1024) and ragged ones (96, 200, 500)
@pytest.mark.parametrize("d", [96, 128, 200, 256, 384, 500, 512, 768, 1024])
def test_batch_stream_rescore_equals_gather(d):
    # tiny and empty jobs between larger ones, a job with long runs of candidates per A row, units of 32
    # candidates that cross job boundaries, planted near pairs
    sizes = [(3, 50), (0, 40), (1, 1), (0, 0), (70, 90), (2, 300), (0, 5), (1500, 1200), (5, 0), (130, 260), (7, 7)]
    jobs_np = make_jobs(11, sizes, d, 0.5 / np.sqrt(d), 1.5 / np.sqrt(d))  # 7 % to 31 % of the pairs
    jobs_dev = to_dev(jobs_np)
    kp, sp, st_p = records({"prec": "bf16"}, jobs_dev)
    kg, sg, st_g = records({"prec": "bf16"}, jobs_dev, pkg.EJOIN_FLAG_GATHER_RESCORE)
    assert len(kp) > 20000
    assert np.array_equal(kp, kg)
    assert np.array_equal(sp, sg)
    assert st_p["launches"] > st_g["launches"]  # the streaming path ran (its sort kernels)
    job = (kp >> 42).astype(np.int64)
    gi = ((kp >> 21) & ((1 << 21) - 1)).astype(np.uint32)
    gj = (kp & ((1 << 21) - 1)).astype(np.uint32)
    check_batch(jobs_np, job, gi, gj, sp.view(np.float32))


def test_batch_stream_rescore_accurate_tier():
    # a wide FP64 band sends many candidates through the accurate tier of both paths
    jobs_np = make_jobs(12, [(400, 500), (90, 30), (1000, 700)], 128, 0.05, 0.12)
    jobs_dev = to_dev(jobs_np)
    kw = {"prec": "bf16", "fp64_band": 0.05}
    kp, sp, st_p = records(kw, jobs_dev)
    kg, sg, st_g = records(kw, jobs_dev, pkg.EJOIN_FLAG_GATHER_RESCORE)
    assert st_p["fp64_rescored"] > 1000 and st_p["fp64_rescored"] == st_g["fp64_rescored"]
    assert np.array_equal(kp, kg) and np.array_equal(sp, sg)


OPS_NP = {"<": np.less, "<=": np.less_equal, ">": np.greater, ">=": np.greater_equal, "==": np.equal,
          "!=": np.not_equal}


def job_selection(rng, n, kind):
    """(device Sel or None, host keep mask) for one side of one job."""
    if kind is None or n == 0:
        return None, np.ones(n, dtype=bool)
    attr = rng.integers(0, 100, n).astype(np.int32)
    bits = None
    keep = np.ones(n, dtype=bool)
    op, c = "<", 0
    if kind in OPS_NP:
        op, c = kind, int(rng.integers(20, 80))
        keep = OPS_NP[op](attr, c)
    elif kind == "none":
        op, c = "<", 0  # attr >= 0: keeps nothing
        keep = np.zeros(n, dtype=bool)
    if kind in ("bits", "attr+bits"):
        b = rng.integers(0, 2, n).astype(bool)
        words = np.zeros((n + 31) // 32, dtype=np.uint32)
        for r in np.nonzero(b)[0]:
            words[r >> 5] |= np.uint32(1) << np.uint32(r & 31)
        bits = torch.from_numpy(words.view(np.int32)).cuda()
        if kind == "attr+bits":
            op, c = ">=", 30
            keep = (attr >= 30) & b
        else:
            keep = b
    a_dev = torch.from_numpy(attr).cuda() if kind != "bits" else None
    return pkg.Sel(a_dev, op, c, bits), keep


def as_oracle_sel(keep):
    # the kept rows as a predicate the oracle evaluates: attr' = 0 for kept rows, 1 otherwise, attr' < 1
    return oracle.Selection(np.where(keep, 0, 1).astype(np.int32), "<", 1)


SEL_KINDS = [("<", None), (None, ">="), ("<=", "=="), ("!=", "bits"), ("attr+bits", ">"), (None, None),
             ("none", "<"), (">", "attr+bits"), ("bits", None), ("==", "!="), ("<", "<")]


def selected_batch(seed, d):
    rng = np.random.default_rng(seed)
    sizes = [(300, 700), (0, 50), (40, 0), (129, 257), (1000, 513), (37, 2000), (256, 256), (5, 900), (777, 31),
             (2000, 1500), (64, 64)]
    jobs_np = make_jobs(seed, sizes, d, 0.5 / np.sqrt(d), 1.5 / np.sqrt(d))
    sels, keeps = [], []
    for (R, S, _), (kr, ks) in zip(jobs_np, SEL_KINDS):
        sr, mr = job_selection(rng, R.shape[0], kr)
        ss, ms = job_selection(rng, S.shape[0], ks)
        sels.append((sr, ss))
        keeps.append((mr, ms))
    return jobs_np, sels, keeps


@pytest.mark.parametrize("prec,d", [("bf16", 96), ("fp8", 128), ("tf32", 64), ("bf16", 384)])
def test_batch_per_job_selections_match_oracle(prec, d):
    jobs_np, sels, keeps = selected_batch(31, d)
    with pkg.Ctx(device=0, prec=prec) as ctx:
        job, gi, gj, gs = pkg.ejoin_batch(ctx, to_dev(jobs_np), graph=True, sels=sels)
    assert len(job) > 1000
    gi, gj = gi.view(np.uint32), gj.view(np.uint32)
    for k, ((R, S, eps), (mr, ms)) in enumerate(zip(jobs_np, keeps)):
        sel = job == k
        oi, oj, os_ = oracle.join(R, S, eps, as_oracle_sel(mr) if len(mr) else None,
                                  as_oracle_sel(ms) if len(ms) else None)
        compare(R, S, eps, gi[sel], gj[sel], gs[sel], oi, oj, os_)
        if sel.any():
            assert mr[gi[sel]].all() and ms[gj[sel]].all()


def test_batch_selections_stream_equals_gather_and_follow_new_attributes():
    jobs_np, sels, keeps = selected_batch(32, 384)
    jobs_dev = to_dev(jobs_np)
    got = {}
    for flags in (0, pkg.EJOIN_FLAG_GATHER_RESCORE):
        with pkg.Ctx(device=0, prec="bf16", flags=flags) as ctx:
            job, gi, gj, gs = pkg.ejoin_batch(ctx, jobs_dev, graph=True, sels=sels)
        key = (job.astype(np.int64) << 42) | (gi.view(np.uint32).astype(np.int64) << 21) | gj.view(np.uint32)
        o = np.argsort(key)
        got[flags] = (key[o], gs[o].view(np.uint32))
    assert np.array_equal(got[0][0], got[pkg.EJOIN_FLAG_GATHER_RESCORE][0])
    assert np.array_equal(got[0][1], got[pkg.EJOIN_FLAG_GATHER_RESCORE][1])
    # a replayed plan evaluates the predicates on the attribute values of each run: the odd rows are given
    # a failing value, so each side keeps the even rows of its former kept set (the sized buffers still fit)
    fail = {"<": 99, "<=": 99, ">": 0, ">=": 0}
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        b = pkg.Batch(ctx, jobs_dev, graph=True, sels=sels)
        b.run()
        n0 = b.wait()
        new_keeps = []
        for (sr, ss), (mr, ms) in zip(sels, keeps):
            nk = []
            for s, m in ((sr, mr), (ss, ms)):
                if s is not None and s.attr is not None:
                    a2 = s.attr.cpu().numpy().copy()
                    a2[1::2] = fail.get(s.op, s.c + 1 if s.op == "==" else s.c)
                    s.attr.copy_(torch.from_numpy(a2))
                    m = m.copy()
                    m[1::2] = False
                nk.append(m)
            new_keeps.append(tuple(nk))
        torch.cuda.synchronize()
        b.run()
        n1 = b.wait()
        job, gi, gj, gs = (x.cpu().numpy() for x in b.result(n1))
        b.close()
    assert n0 > n1 > 0
    gi, gj = gi.view(np.uint32), gj.view(np.uint32)
    for k, ((R, S, eps), (mr, ms)) in enumerate(zip(jobs_np, new_keeps)):
        sel = job == k
        oi, oj, os_ = oracle.join(R, S, eps, as_oracle_sel(mr) if len(mr) else None,
                                  as_oracle_sel(ms) if len(ms) else None)
        compare(R, S, eps, gi[sel], gj[sel], gs[sel], oi, oj, os_)
