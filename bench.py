#!/usr/bin/env python
"""Benchmark of the E-join tensor-join hot path on one GB300 (or N replicas).

One step = one full pass of the path over one batch of synthetic input:
selection + normalisation of R and S, the blocked similarity contraction
fused with the threshold and compaction, the exact re-score, and the pair
count read-back (one ejoin_threshold call through the C ABI).

Default workload (the metric's configuration): R = 1,000,000 and S = 100,000
rows, d = 300, clustered unit vectors (1000 centres, ~0.3 rad spread), the
relational predicate attr < 100 on R (10 % selectivity) pushed into the path,
eps = 0.85, BF16 contraction with FP32/FP64 re-score of the guard band.

Prints ONE JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "E-join pair comparisons/sec at exact-set match vs FP64; % of tensor peak"
METRIC_TOPK = "top-k join pair comparisons/sec (top k within 1e-5 of FP64); % of tensor peak"
UNIT = "pairs/s"
CONTRACT_SOURCES = ["sim_tc.cu", "sim_simt.cu", "ejoin_internal.cuh"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float) -> float:
    """The maximum of x over the ranks of the default process group (x itself without one): the step time
    of a run of N replicas is that of its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            m = json.load(f)
        return {"hbm_gbs": m["hbm_gbs"], "bf16_tflops": m["bf16_tflops"],
                "bf16_tflops_sustained": m.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


ESEL_SOURCES = ["esel.cu", "ejoin_internal.cuh"]


def contract_source_sha(sources=None):
    h = hashlib.sha256()
    for f in sources or CONTRACT_SOURCES:
        with open(os.path.join(ROOT, "paper_2312_01476_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str, sources=None):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's sources still hash to the
    recorded value."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    e = t.get(kernel_key)
    if not e or e.get("source_sha") != contract_source_sha(sources):
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = os.path.join("/tmp", f"ejoin_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx = max(mx, float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(args, seed_offset=0):
    import ejoin_inputs as inputs
    if args.workload == "c2":
        w = inputs.c2_clustered_selection(threads=os.cpu_count() or 8)
    elif args.workload == "c2-capture":
        # same structure at 30 % of R: the size used for full ncu captures
        w = inputs.c2_clustered_selection(nR=300_000, nS=100_000, threads=os.cpu_count() or 8)
    elif args.workload == "c1":
        w = inputs.c1_planted()
    elif args.workload == "c3":
        w = inputs.c3_clustered_selfjoin(threads=os.cpu_count() or 8)
    elif args.workload == "c3-capture":
        w = inputs.c3_clustered_selfjoin(n=200_000, threads=os.cpu_count() or 8)
    elif args.workload in ("top1", "top32"):
        w = inputs.topk_clustered_selection(sel_c=args.sel_pct, threads=os.cpu_count() or 8)
    elif args.workload in ("top1-capture", "top32-capture"):
        w = inputs.topk_clustered_selection(nS=300_000, sel_c=args.sel_pct, threads=os.cpu_count() or 8)
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    return w


def cpu_oracle_sample(w, target_s: float, threads: int):
    """Time the FP64 oracle on selected R rows x all S rows, about target_s seconds of work."""
    import oracle
    sel = np.nonzero(w.attrR < w.cR)[0] if w.attrR is not None else np.arange(w.R.shape[0])
    selR = oracle.Selection(w.attrR, w.opR, w.cR) if w.attrR is not None else None
    n_s = w.S.shape[0]
    # probe twice: the first call also pays for the (serial) norms of S
    k = 32
    for _ in range(2):
        t = time.perf_counter()
        oracle.join(w.R, w.S, w.eps, selR, rows=sel[:k], threads=threads)
        dt = max(time.perf_counter() - t, 1e-3)
        k = int(min(len(sel), max(8, 0.9 * target_s / dt * k)))
        if dt > 0.2 * target_s:
            break
    rows = sel[:k]
    t = time.perf_counter()
    oracle.join(w.R, w.S, w.eps, selR, rows=rows, threads=threads)
    dt = time.perf_counter() - t
    return {"value": k * n_s / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{k} selected R rows x all {n_s} S rows (FP64, extrapolated pairs/s)",
            "seconds": round(dt, 3)}


def topk_of(workload: str) -> int:
    return 32 if workload.startswith("top32") else 1


def cpu_oracle_topk_sample(w, k: int, target_s: float, threads: int):
    """Time the FP64 oracle's top-k on R rows x all kept S rows, about target_s seconds of work."""
    import oracle
    selS = oracle.Selection(w.attrS, w.opS, w.cS) if w.attrS is not None else None
    n_s = int((w.attrS < w.cS).sum()) if w.attrS is not None else w.S.shape[0]
    m = 16
    for _ in range(2):
        t = time.perf_counter()
        oracle.topk(w.R, w.S, k, None, selS, rows=np.arange(m), threads=threads)
        dt = max(time.perf_counter() - t, 1e-3)
        m = int(min(w.R.shape[0], max(8, 0.9 * target_s / dt * m)))
        if dt > 0.2 * target_s:
            break
    t = time.perf_counter()
    oracle.topk(w.R, w.S, k, None, selS, rows=np.arange(m), threads=threads)
    dt = time.perf_counter() - t
    return {"value": m * n_s / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"top-{k} of {m} R rows over all {n_s} kept S rows (FP64, extrapolated pairs/s)",
            "seconds": round(dt, 3)}


def reference_sampled(args, threads):
    """The oracle on a bounded sample of the batched (c4), learned (c5) and E-selection workloads, whose
    full inputs are generated on the device: same recipes, a few rows of R against a block of S (or the
    queries), pairs/s extrapolated to the full step."""
    import oracle
    import ejoin_inputs as inputs
    if args.workload == "esel":
        d, m, eps, seed = 768, 32, 0.9, inputs.seed_for(7)
        centres = inputs.sphere_centres(20_000, d, seed)
        R = inputs.clustered(20_000, d, centres, inputs.THETA_768, seed + 10, threads)
        S = inputs.clustered(m, d, centres, inputs.THETA_768, seed + 20, threads)
        full, metric = 10_000_000 * m, METRIC_ESEL
        name = "E-selection: R = 10000000 x 768 clustered rows (20,000 centres), 32 queries, eps=0.9"
        sample = "20,000 rows x 32 queries (FP64)"
    elif args.workload == "c4":
        d, eps, seed = 384, 0.875, inputs.seed_for(4)
        centres = inputs.sphere_centres(1000, d, seed)
        R = inputs.clustered(64, d, centres, 0.3, seed + 1, threads)
        S = inputs.clustered(20_000, d, centres, 0.3, seed + 2, threads)
        sizes, _ = inputs.c4_batch_sizes()
        full, metric = int((sizes[:, 0] * sizes[:, 1]).sum()), METRIC
        name = "batched joins: 512 jobs, lognormal sizes (median 20,000), d=384"
        sample = "64 rows x 20,000 rows of a median-size job (FP64)"
    else:  # c5
        d, eps, seed = 768, 0.9, inputs.seed_for(5)
        centres = inputs.sphere_centres(20_000, d, seed)
        S = inputs.clustered(200_000, d, centres, inputs.THETA_768, seed + 10, threads)
        R = S[:8]
        full, metric = 4_000_000 ** 2, METRIC
        name = "clustered self-join n=4000000 d=768 eps=0.90"
        sample = "8 rows x 200,000 rows of the same recipe (FP64)"
    vals = []
    for step in range(args.warmup + args.steps):
        t = time.perf_counter()
        n_calls = 0
        while True:
            oracle.join(R, S, eps, threads=threads)
            n_calls += 1
            if time.perf_counter() - t >= min(args.ref_step_s, 5.0):
                break
        dt = time.perf_counter() - t
        if step >= args.warmup:
            vals.append(n_calls * R.shape[0] * S.shape[0] / dt)
    return name, metric, full, statistics.median(vals), sample


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload in ("c4", "c5", "esel"):
        threads = os.cpu_count() or 1
        name, metric, full, v, sample = reference_sampled(args, threads)
        out = {"impl": "reference", "metric": metric, "value": v, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": full / v * 1e3, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": name, "pairs_per_step": full},
               "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
               "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return
    w = make_workload(args)
    if args.workload.startswith("top"):
        threads = os.cpu_count() or 1
        k = topk_of(args.workload)
        vals = [cpu_oracle_topk_sample(w, k, args.ref_step_s, threads) for _ in range(args.warmup + args.steps)]
        vals = vals[args.warmup:]
        v = statistics.median([r["value"] for r in vals])
        pairs = w.R.shape[0] * int((w.attrS < w.cS).sum())
        out = {"impl": "reference", "metric": METRIC_TOPK, "value": v, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": pairs / v * 1e3, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": w.name, "pairs_per_step": pairs, "d": int(w.R.shape[1])},
               "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": vals[0]["sample"]},
               "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return
    threads = os.cpu_count() or 1
    n_sel_r = int((w.attrR < w.cR).sum()) if w.attrR is not None else w.R.shape[0]
    vals = []
    for s in range(args.warmup + args.steps):
        r = cpu_oracle_sample(w, args.ref_step_s, threads)
        if s >= args.warmup:
            vals.append(r)
    v = statistics.median([r["value"] for r in vals])
    ms = n_sel_r * w.S.shape[0] / v * 1e3
    # the oracle runs on a bounded sample of each step's pairs: ms_per_step is extrapolated from the sampled
    # pairs/s to the full step (the GPU arm's keys are given too; those that describe a GPU result are null)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "extrapolated": True, "sampled_seconds_per_step": round(statistics.median([r["seconds"] for r in vals]), 3),
           "config": {"workload": w.name, "pairs_per_step": n_sel_r * w.S.shape[0], "d": int(w.R.shape[1]),
                      "n_sel_r": n_sel_r, "n_sel_s": int(w.S.shape[0]), "result_pairs": None, "candidates": None,
                      "fp64_rescored": None, "band": None, "symmetric_self_join": False,
                      "l2": "not applicable (host cores)", "parallelism": "FP64 oracle, OpenMP over the host cores"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": vals[0]["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ejoin(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2312_01476_gb300 as pkg

    w = make_workload(args)
    if args.prec == "f32" and args.workload == "c3":
        # the CUDA-core FP32 path needs minutes for the full 2M x 2M self-join: join the first
        # 100,000 rows with all rows instead (stated in config.workload)
        w.R = w.R[:100_000]
        w.self_join = False
        w.name += " (R = first 100,000 rows, fp32 CUDA-core path)"
    d = int(w.R.shape[1])
    R = torch.from_numpy(w.R).cuda()
    S = R if w.self_join else torch.from_numpy(w.S).cuda()
    attr = torch.from_numpy(w.attrR).cuda() if w.attrR is not None else None
    selR = pkg.Sel(attr, w.opR, w.cR) if attr is not None else None
    fp64_band = 2e-3 if args.workload.startswith("c3") else -1.0
    flags = pkg.EJOIN_FLAG_TIMING | (pkg.EJOIN_FLAG_GATHER_RESCORE if args.gather_rescore else 0)
    ctx = pkg.Ctx(device=local, prec=args.prec, flags=flags, group_m=args.group_m, fp64_band=fp64_band)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    for _ in range(args.warmup):
        res = pkg.ejoin_threshold(ctx, R, S, w.eps, selR)
    torch.cuda.synchronize()
    st0 = pkg.ejoin_last_stats(ctx)
    pairs_per_step = int(st0["n_sel_r"]) * int(st0["n_sel_s"])

    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    contract_ms, launches, stage = [], 0, {"normalize": [], "rescore": []}
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # L2 flush between steps (not timed)
        ev[k][0].record()
        res = pkg.ejoin_threshold(ctx, R, S, w.eps, selR)
        ev[k][1].record()
        st = pkg.ejoin_last_stats(ctx)
        contract_ms.append(st["ms_contract"])
        stage["normalize"].append(st["ms_normalize"])
        stage["rescore"].append(st["ms_rescore"])
        launches += int(st["launches"])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    ms = max_over_ranks(ms)
    n_pairs = int(res.count)
    value = world * pairs_per_step / (ms * 1e-3)

    pk = peaks()
    c_ms = statistics.mean(contract_ms)
    # FLOPs the contraction performs for the step's logical pairs: a self-join on the tensor cores is
    # evaluated on the upper triangle only, so it gets no credit for the mirrored half
    symmetric = w.self_join and args.prec != "f32"
    n_sel = int(st0["n_sel_r"])
    flop = 2.0 * d * (n_sel * (n_sel + 1) // 2 if symmetric else pairs_per_step)
    if args.prec == "f32":
        peak, peak_note = None, "fp32 SIMT"
    else:
        peak, peak_note = tensor_peak(args.prec, c_ms)
    kernel_key = f"sim_tc_{args.prec}_{args.workload}" if args.prec != "f32" else f"sim_simt_{args.workload}"
    achieved = flop / (c_ms * 1e-3) / 1e12
    roofline = {"kernel": kernel_key, "bound": "tensor", "achieved": round(achieved, 2),
                "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4) if peak else None,
                "peak_note": peak_note, "traffic": recorded_traffic(kernel_key),
                "flop_per_launch": flop, "ms_per_launch": round(c_ms, 4)}

    # end to end through the host-memory entry point (pinned buffers, copies timed)
    e2e = None
    if not args.no_e2e:
        Rp = torch.from_numpy(w.R).pin_memory()
        Sp = Rp if w.self_join else torch.from_numpy(w.S).pin_memory()
        Ap = torch.from_numpy(w.attrR).pin_memory() if w.attrR is not None else None
        cap = n_pairs + (1 << 20)
        out = torch.empty(cap * 12, dtype=torch.uint8).pin_memory().numpy().view(pkg.PAIR_DTYPE)
        hsel = pkg.Sel(Ap.numpy(), w.opR, w.cR) if Ap is not None else None
        for _ in range(2):
            pkg.ejoin_threshold_host(ctx, Rp.numpy(), Sp.numpy(), w.eps, hsel, out=out)
        e_ms, h2d_ms = [], []
        for k in range(max(3, args.steps // 2)):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            pr, cnt = pkg.ejoin_threshold_host(ctx, Rp.numpy(), Sp.numpy(), w.eps, hsel, out=out)
            b.record()
            b.synchronize()
            e_ms.append(a.elapsed_time(b))
            h2d_ms.append(pkg.ejoin_last_stats(ctx)["ms_h2d"])
        em = statistics.mean(e_ms)
        hst = pkg.ejoin_last_stats(ctx)
        # bytes that crossed the host link: with pinned inputs the kernels read only the predicate columns and
        # the kept rows in place; otherwise the inputs are copied whole
        e2e = {"value": world * pairs_per_step / (em * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(hst["h2d_bytes"]),
               "d2h_bytes_per_step": int(cnt * 12 + 8), "ms_per_step": round(em, 3),
               "inputs_read_in_place": bool(hst["host_in_place"]),
               "ms_h2d_copies": round(statistics.mean(h2d_ms), 3)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w, args.cpu_s, os.cpu_count() or 1)
    large = None
    if args.workload == "c2" and args.prec == "bf16" and not args.no_large_join:
        del R, S
        torch.cuda.empty_cache()
        large = measure_large_join(args, local)
    forms = None
    if args.workload == "c2" and args.prec == "bf16" and not args.no_forms and world == 1:
        # the batched and the learned form on their own workloads, each beside the plain FP32 path on the
        # same GPU (summaries of the lines `--workload c4` and `--workload c5` print)
        forms = measure_forms(args)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
               "config": {"workload": w.name, "pairs_per_step": pairs_per_step, "d": d,
                          "n_sel_r": int(st0["n_sel_r"]), "n_sel_s": int(st0["n_sel_s"]),
                          "result_pairs": n_pairs, "candidates": int(st0["candidates"]),
                          "fp64_rescored": int(st0["fp64_rescored"]), "band": st0["band"],
                          "symmetric_self_join": symmetric,
                          "l2": "256 MB buffer written between timed steps (untimed)",
                          "parallelism": f"{world} independent replica(s)"},
               "stages_ms": {"normalize": round(statistics.mean(stage["normalize"]), 4),
                             "contract": round(c_ms, 4), "rescore": round(statistics.mean(stage["rescore"]), 4)},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clocks, "large_join": large, "forms": forms}
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_forms(args):
    """Summaries of the batched form (c4: 512 joins, graph replay, 5 timed steps) and of the learned form
    (c5: the 4M-row self-join with learned tile pruning, 2 timed steps), each with the plain FP32 CUDA-core
    path measured on the same GPU."""
    import argparse
    ba = argparse.Namespace(**{**vars(args), "workload": "c4", "steps": 5, "warmup": 3, "prec": "bf16"})
    b = run_batch(ba, emit=False)
    la = argparse.Namespace(**{**vars(args), "workload": "c5", "steps": 2, "warmup": 3, "prec": "bf16"})
    lr = run_learned(la, emit=False)
    bl = b["baselines"]
    return {
        "batched": {"workload": b["config"]["workload"], "value": b["value"], "unit": b["unit"],
                    "ms_per_step": b["ms_per_step"], "steps": b["steps"], "warmup": b["warmup"],
                    "latency_ms": b["latency_ms"], "roofline": b["roofline"], "clocks": b["clocks"],
                    "stages_ms": {"normalize": b["config"]["ms_normalize"], "contract": b["config"]["ms_contract"],
                                  "rescore": b["config"]["ms_rescore"]},
                    "sequential_calls_pairs_per_s": bl["sequential_calls_pairs_per_s"],
                    "fp32_cuda_cores_pairs_per_s": bl["fp32_cuda_cores_pairs_per_s"], "fp32_sample": bl["fp32_sample"],
                    "speedup_vs_fp32_cuda_cores": b["value"] / bl["fp32_cuda_cores_pairs_per_s"]},
        "learned": {"workload": lr["config"]["workload"], "value": lr["value"], "unit": lr["unit"],
                    "ms_per_step": lr["ms_per_step"], "steps": lr["steps"], "warmup": lr["warmup"],
                    "recall": lr["recall"], "recall_est": lr["pruned"]["recall_est"],
                    "plain_bf16_ms_per_step": lr["plain_bf16"]["ms_per_step"],
                    "speedup_vs_plain_bf16": lr["speedup_vs_plain_bf16"],
                    "fp32_cuda_cores_pairs_per_s": lr["plain_fp32_cuda_cores"]["pairs_per_s"],
                    "fp32_sample": lr["plain_fp32_cuda_cores"]["sample"],
                    "speedup_vs_fp32_cuda_cores": lr["speedup_vs_plain_fp32"],
                    "stages_ms": {k: lr["pruned"][k] for k in ("ms_prepare", "ms_bound", "ms_contract", "ms_rescore")}},
    }


def measure_large_join(args, local):
    """The large threshold join the tensor-peak target is stated for: the 2,000,000-row clustered
    self-join at d = 768 (eps = 0.95, FP64 tier band 2e-3), BF16, 1 warm-up and 2 timed steps with the
    L2 flushed between them; its own stages, roofline (sustained peak: the launch runs ~2 s under the
    power cap) and clocks."""
    import torch
    import paper_2312_01476_gb300 as pkg
    import ejoin_inputs as inputs
    w = inputs.c3_clustered_selfjoin(threads=os.cpu_count() or 8)
    X = torch.from_numpy(w.R).cuda()
    d = int(w.R.shape[1])
    ctx = pkg.Ctx(device=local, prec="bf16", flags=pkg.EJOIN_FLAG_TIMING, fp64_band=2e-3)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    pkg.ejoin_threshold(ctx, X, X, w.eps)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ms, contract, rescore = [], [], []
    for k in range(2):
        flush.fill_(k & 0xFF)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = pkg.ejoin_threshold(ctx, X, X, w.eps)
        z.record()
        z.synchronize()
        ms.append(a.elapsed_time(z))
        st = pkg.ejoin_last_stats(ctx)
        contract.append(st["ms_contract"])
        rescore.append(st["ms_rescore"])
    clocks = sampler.stop()
    n = X.shape[0]
    step = statistics.mean(ms)
    c_ms = statistics.mean(contract)
    flop = 2.0 * d * (n * (n + 1) // 2)  # the upper triangle the symmetric contraction evaluates
    peak, note = tensor_peak("bf16", c_ms)
    out = {"workload": w.name, "dtype": "bf16", "pairs_per_step": n * n, "value": n * n / (step * 1e-3),
           "unit": UNIT, "ms_per_step": round(step, 2), "steps": 2, "warmup": 1, "result_pairs": int(res.count),
           "fp64_rescored": int(st["fp64_rescored"]),
           "stages_ms": {"normalize": round(st["ms_normalize"], 3), "contract": round(c_ms, 2),
                         "rescore": round(statistics.mean(rescore), 2)},
           "roofline": {"kernel": "sim_tc_bf16_c3", "bound": "tensor", "achieved": round(flop / (c_ms * 1e-3) / 1e12, 2),
                        "peak": peak, "unit": "TFLOP/s", "frac": round(flop / (c_ms * 1e-3) / 1e12 / peak, 4),
                        "peak_note": note, "flop_per_launch": flop, "ms_per_launch": round(c_ms, 2),
                        "traffic": recorded_traffic("sim_tc_bf16_c3")},
           "clocks": clocks, "l2": "256 MB buffer written between timed steps (untimed)"}
    ctx.close()
    del X, res
    torch.cuda.empty_cache()
    return out


def tensor_peak(prec, contract_ms):
    """The roofline denominator for a contraction of this precision (TFLOP/s) and its note: a launch
    of half a second or more runs under the power cap, so it is compared with the sustained peak."""
    pk = peaks()
    sustained = contract_ms > 500.0 and pk.get("bf16_tflops_sustained")
    base = pk["bf16_tflops_sustained"] if sustained else pk["bf16_tflops"]
    kind = "sustained" if sustained else "burst"
    if prec == "bf16":
        return base, f"bf16 dense {kind}, {pk['source']}"
    if prec == "fp8":
        return 2 * base, f"2 x bf16 {kind} ({pk['source']}, nominal fp8/bf16 ratio)"
    return 0.5 * base, f"0.5 x bf16 {kind} ({pk['source']}, nominal tf32/bf16 ratio)"


def run_topk(args):
    """Top-k join condition (k = 1 or 32): 10,000 query rows against 1,000,000 rows under a pushed-down
    S predicate; one step = one ejoin_topk call (selection, normalisation, the two contraction passes,
    the FP32 re-score and per-row selection of the candidates, k records per query)."""
    import torch
    import paper_2312_01476_gb300 as pkg
    if args.prec == "f32":
        raise SystemExit("top-k runs on the tensor cores only (bf16, fp8, tf32)")
    k = topk_of(args.workload)
    w = make_workload(args)
    d = int(w.R.shape[1])
    R = torch.from_numpy(w.R).cuda()
    S = torch.from_numpy(w.S).cuda()
    A = torch.from_numpy(w.attrS).cuda()
    selS = pkg.Sel(A, w.opS, w.cS)
    ctx = pkg.Ctx(device=0, prec=args.prec, flags=pkg.EJOIN_FLAG_TIMING, group_m=args.group_m)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        res = pkg.ejoin_topk(ctx, R, S, k, None, selS)
    torch.cuda.synchronize()
    st0 = pkg.ejoin_last_stats(ctx)
    pairs = int(st0["n_sel_r"]) * int(st0["n_sel_s"])
    sampler = ClockSampler(0)
    sampler.start()
    step_ms, cms, stage, launches = [], [], {"normalize": [], "rescore": []}, 0
    torch.cuda.synchronize()
    for step in range(args.steps):
        flush.fill_(step & 0xFF)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = pkg.ejoin_topk(ctx, R, S, k, None, selS)
        z.record()
        st = pkg.ejoin_last_stats(ctx)
        cms.append(st["ms_contract"])
        stage["normalize"].append(st["ms_normalize"])
        stage["rescore"].append(st["ms_rescore"])
        launches += int(st["launches"])
        z.synchronize()
        step_ms.append(a.elapsed_time(z))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = statistics.mean(step_ms)
    c_ms = statistics.mean(cms)
    # executed FLOPs, 2 d per evaluated pair: BF16/TF32 top-1 evaluates every kept pair once (one pass);
    # k > 1 and e4m3 add the first pass over every stride-th 256-column tile (stride 8 while at least 4k
    # tiles remain)
    two_pass = k > 1 or args.prec == "fp8"
    passes = 2 if two_pass else 1
    flop = 2.0 * d * pairs
    if two_pass:
        n_s = int(st0["n_sel_s"])
        tiles = -(-n_s // 256)
        stride = max(1, min(8, tiles // (4 * k)))
        flop += 2.0 * d * int(st0["n_sel_r"]) * min(n_s, -(-tiles // stride) * 256)
    peak, note = tensor_peak(args.prec, c_ms / passes)
    achieved = flop / (c_ms * 1e-3) / 1e12
    kernel_key = f"sim_tc_top_{args.prec}_{args.workload}"
    roofline = {"kernel": kernel_key + (" (passes 0 + 1)" if two_pass else " (single pass)"), "bound": "tensor",
                "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "peak_note": note + ("; both passes and the threshold kernel between them" if two_pass else ""),
                "traffic": recorded_traffic(kernel_key), "flop_per_step": flop, "ms_contract": round(c_ms, 4)}
    # end to end through the public API: pinned host inputs copied in, the records copied out
    e2e = None
    if not args.no_e2e:
        Rp, Sp, Ap = (torch.from_numpy(a).pin_memory() for a in (w.R, w.S, w.attrS))
        out = torch.empty((w.R.shape[0] * k, 3), dtype=torch.int32).pin_memory()
        e_ms = []
        for step in range(2 + max(3, args.steps // 2)):
            flush.fill_(step & 0xFF)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            Rd, Sd, Ad = Rp.cuda(non_blocking=True), Sp.cuda(non_blocking=True), Ap.cuda(non_blocking=True)
            r = pkg.ejoin_topk(ctx, Rd, Sd, k, None, pkg.Sel(Ad, w.opS, w.cS))
            n = r.count
            out[:n].copy_(torch.stack([r.i, r.j, r.sim.view(torch.int32)], 1), non_blocking=True)
            z.record()
            z.synchronize()
            if step >= 2:
                e_ms.append(a.elapsed_time(z))
            del Rd, Sd, Ad
        em = statistics.mean(e_ms)
        e2e = {"value": pairs / (em * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(w.R.nbytes + w.S.nbytes +
                                                                                      w.attrS.nbytes),
               "d2h_bytes_per_step": int(n * 12 + 8), "ms_per_step": round(em, 3)}
    cpu = None if args.no_cpu_baseline else cpu_oracle_topk_sample(w, k, args.cpu_s, os.cpu_count() or 1)
    out = {"metric": METRIC_TOPK, "value": pairs / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
           "config": {"workload": w.name + f", k={k}", "k": k, "pairs_per_step": pairs, "d": d,
                      "n_sel_r": int(st0["n_sel_r"]),
                      "n_sel_s": int(st0["n_sel_s"]), "records": int(res.count),
                      "candidates": int(st0["candidates"]), "band": st0["band"],
                      "l2": "256 MB buffer written between timed steps (untimed)",
                      "parallelism": "1 replica"},
           "stages_ms": {"normalize": round(statistics.mean(stage["normalize"]), 4), "contract": round(c_ms, 4),
                         "rescore": round(statistics.mean(stage["rescore"]), 4)},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out), flush=True)
    ctx.close()


METRIC_ESEL = "E-selection row-query comparisons/sec at exact-set match vs FP64; % of HBM bandwidth"


def run_eselect(args):
    """ℰ-selection scan: 10,000,000 x 768 FP32 rows against 32 query rows at eps = 0.9; one step = one
    ejoin_eselect call (query normalisation, the TF32 scan reading R once, the exact re-score)."""
    import torch
    import ejoin_inputs as inputs
    import paper_2312_01476_gb300 as pkg
    R, Q, eps = inputs.eselect_workload(n=args.esel_rows)
    n, d = R.shape
    m = Q.shape[0]
    ctx = pkg.Ctx(device=0, flags=pkg.EJOIN_FLAG_TIMING)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        res = pkg.ejoin_eselect(ctx, R, Q, eps)
    torch.cuda.synchronize()
    st0 = pkg.ejoin_last_stats(ctx)
    sampler = ClockSampler(0)
    sampler.start()
    step_ms, scan_ms, launches = [], [], 0
    for step in range(args.steps):
        flush.fill_(step & 0xFF)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        res = pkg.ejoin_eselect(ctx, R, Q, eps)
        z.record()
        st = pkg.ejoin_last_stats(ctx)
        scan_ms.append(st["ms_contract"])
        launches += int(st["launches"])
        z.synchronize()
        step_ms.append(a.elapsed_time(z))
    clocks = sampler.stop()
    ms = statistics.mean(step_ms)
    s_ms = statistics.mean(scan_ms)
    pk = peaks()
    algo_bytes = n * d * 4  # every row of R read once; the queries come from L2
    achieved = algo_bytes / (s_ms * 1e-3) / 1e9
    roofline = {"kernel": "esel_kernel", "bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4),
                "peak_note": f"STREAM-style copy, {pk['source']}", "traffic": recorded_traffic("esel_kernel_esel", ESEL_SOURCES),
                "bytes_per_launch": algo_bytes, "ms_per_launch": round(s_ms, 4)}
    e2e = None
    if not args.no_e2e:
        Rp = R.cpu().pin_memory()
        Qp = Q.cpu().pin_memory()
        e_ms = []
        for step in range(2 + 3):
            flush.fill_(step & 0xFF)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            Rd, Qd = Rp.cuda(non_blocking=True), Qp.cuda(non_blocking=True)
            r = pkg.ejoin_eselect(ctx, Rd, Qd, eps)
            host = torch.stack([r.i, r.j, r.sim.view(torch.int32)], 1).cpu()
            z.record()
            z.synchronize()
            if step >= 2:
                e_ms.append(a.elapsed_time(z))
            del Rd, Qd
        em = statistics.mean(e_ms)
        e2e = {"value": n * m / (em * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(n * d * 4 + m * d * 4),
               "d2h_bytes_per_step": int(host.numel() * 4), "ms_per_step": round(em, 3)}
        del Rp
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        Qh = Q.cpu().numpy()
        k = 20_000
        Rs = R[:k].cpu().numpy()
        t = time.perf_counter()
        oracle.join(Rs, Qh, eps, threads=os.cpu_count() or 1)
        dt = time.perf_counter() - t
        cpu = {"value": k * m / dt, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"first {k} rows x all {m} queries (FP64)", "seconds": round(dt, 3)}
    out = {"metric": METRIC_ESEL, "value": n * m / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "tf32", "data": "synthetic",
           "config": {"workload": f"E-selection: R = {n} x {d} clustered rows (20,000 centres), {m} queries, eps={eps}",
                      "rows": n, "queries": m, "d": d, "result_pairs": int(res.count),
                      "candidates": int(st0["candidates"]), "band": st0["band"], "in_place_scan": bool(st0["fused"]),
                      "l2": "inputs (30.7 GB) larger than L2; 256 MB buffer written between timed steps",
                      "parallelism": "1 replica"},
           "stages_ms": {"queries": round(st0["ms_normalize"], 4), "scan": round(s_ms, 4),
                         "rescore": round(st0["ms_rescore"], 4)},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(out), flush=True)
    ctx.close()


def run_batch(args, emit=True):
    """512 independent joins (lognormal sizes, per-job eps) in one persistent launch, replayed from a
    CUDA graph; reports the batch latency p50/p99 and pairs/s."""
    import torch
    import ejoin_inputs as inputs
    import paper_2312_01476_gb300 as pkg
    d = 384
    sizes, eps = inputs.c4_batch_sizes(n_jobs=args.batch_jobs)
    centres = torch.from_numpy(inputs.sphere_centres(1000, d, inputs.seed_for(4))).cuda()
    jobs = []
    for k, ((nr, ns), e) in enumerate(zip(sizes.tolist(), eps.tolist())):
        R = inputs.clustered_torch(nr, d, centres, 0.3, inputs.seed_for(4) * 10000 + 2 * k)
        S = inputs.clustered_torch(ns, d, centres, 0.3, inputs.seed_for(4) * 10000 + 2 * k + 1)
        jobs.append((R, S, float(e)))
    torch.cuda.synchronize()
    ctx = pkg.Ctx(device=0, prec=args.prec, flags=pkg.EJOIN_FLAG_TIMING)
    t0 = time.perf_counter()
    b = pkg.Batch(ctx, jobs, graph=True, autotune=True)
    plan_s = time.perf_counter() - t0
    info = b.info()
    for _ in range(args.warmup):
        b.run()
    n_pairs = b.wait()
    sampler = ClockSampler(0)
    sampler.start()
    lat = []
    for _ in range(args.steps):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        b.run()
        z.record()
        z.synchronize()
        lat.append(a.elapsed_time(z))
    n_pairs = b.wait()
    clocks = sampler.stop()
    launches_per_run = int(pkg.ejoin_last_stats(ctx)["launches"])
    logical = int((sizes[:, 0] * sizes[:, 1]).sum())

    # baselines: the same joins one ejoin_threshold call at a time (BF16), and the plain FP32
    # CUDA-core path on every 16th job (pairs/s extrapolated from that sample)
    def seq(prec, ks):
        with pkg.Ctx(device=0, prec=prec) as c1:
            R, S, e = jobs[ks[0]]
            pkg.ejoin_threshold(c1, R, S, e)  # warm-up
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for k in ks:
                R, S, e = jobs[k]
                pkg.ejoin_threshold(c1, R, S, e)
            z.record()
            z.synchronize()
            return a.elapsed_time(z), int(sum(sizes[k, 0] * sizes[k, 1] for k in ks))
    seq_ms, _ = seq(args.prec, list(range(len(jobs))))
    f32_ms, f32_pairs = seq("f32", list(range(0, len(jobs), 16)))
    baselines = {"sequential_calls_ms": round(seq_ms, 2), "sequential_calls_pairs_per_s": logical / (seq_ms * 1e-3),
                 "fp32_cuda_cores_pairs_per_s": f32_pairs / (f32_ms * 1e-3),
                 "fp32_sample": "every 16th job (%d jobs, %d pairs), one call each" % (len(range(0, len(jobs), 16)),
                                                                                       f32_pairs)}
    pk = peaks()
    flop = 2.0 * d * logical
    lat_s = np.array(lat) / 1e3
    out = {"metric": METRIC, "value": logical / float(np.mean(lat_s)), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(float(np.mean(lat)), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
           "data": "synthetic",
           "config": {"workload": f"batched joins: {args.batch_jobs} jobs, lognormal sizes (median 20,000, sigma 1, clipped "
                                  "[1,000, 200,000]), d=384, clustered (1000 centres, 0.3 rad), eps ~ U[0.8, 0.95]",
                      "pairs_per_batch": logical, "result_pairs": int(n_pairs), "plan_seconds": round(plan_s, 2),
                      **{k: v for k, v in info.items()}},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "min": float(np.min(lat)), "max": float(np.max(lat))},
           "roofline": {"bound": "tensor", "achieved_whole_batch": round(flop / float(np.mean(lat_s)) / 1e12, 2),
                        "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                        "frac": round(flop / float(np.mean(lat_s)) / 1e12 / pk["bf16_tflops"], 4),
                        "note": "whole batch (normalise + contraction + re-score) per replay"},
           "gpu_launches": launches_per_run * args.steps, "clocks": clocks, "baselines": baselines}
    if emit:
        print(json.dumps(out), flush=True)
    b.close()
    ctx.close()
    del jobs, b
    torch.cuda.empty_cache()
    return out


def run_learned(args, emit=True):
    """4M-row self-join with learned tile pruning against the plain BF16 join, which checks its result."""
    import torch
    import ejoin_inputs as inputs
    import paper_2312_01476_gb300 as pkg
    from paper_2312_01476_gb300 import ejoin as E
    if args.c5_rows == 4_000_000:
        w = inputs.c5_learned(threads=os.cpu_count() or 8)
    else:  # a smaller case of the same shape: groups of ~200 rows
        w = inputs.c5_learned(n=args.c5_rows, n_clusters=max(1, args.c5_rows // 200), threads=os.cpu_count() or 8)
    d = int(w.R.shape[1])
    X = torch.from_numpy(w.R).cuda()
    Xtr = torch.from_numpy(w.extra["train"]).cuda()
    Xcal = torch.from_numpy(w.extra["calib"]).cuda()
    ctx = pkg.Ctx(device=0, prec="bf16", flags=pkg.EJOIN_FLAG_TIMING)
    sk = E.Sketch(ctx, d, 256, 64)
    # training and calibration in the library: labels from the exact join of a held-out sample, 10M pairs,
    # 3 epochs, eps_sketch for recall 0.999 on a second held-out sample
    eps_sk, train_rep = E.ejoin_sketch_train(sk, Xtr, Xcal, w.eps, n_pairs=10_000_000, epochs=3, batch=65536,
                                             lr=2e-3, recall=0.999, seed=inputs.seed_for(5), init=True)

    def timed(fn, steps, warm):
        for _ in range(warm):
            r = fn()
        ms = []
        for _ in range(steps):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            r = fn()
            z.record()
            z.synchronize()
            ms.append(a.elapsed_time(z))
        return r, float(np.mean(ms))

    (res_p, st_p), ms_pruned = timed(lambda: E.ejoin_threshold_pruned(ctx, sk, X, X, w.eps, eps_sk),
                                     max(2, args.steps), max(3, args.warmup))
    n_pruned = res_p.count
    pruned_sample = None
    rows = np.sort(np.random.default_rng(5).choice(X.shape[0], 16, replace=False))
    gi, gj = res_p.i.cpu().numpy().view(np.uint32), res_p.j.cpu().numpy().view(np.uint32)
    keep = np.isin(gi, rows)
    pruned_sample = set(zip(gi[keep].tolist(), gj[keep].tolist()))
    del res_p
    # the library's sampled recall estimate (an extra call, outside the timed region)
    _, st_est = E.ejoin_threshold_pruned(ctx, sk, X, X, w.eps, eps_sk, recall_est=True)
    st_p["recall_est"] = st_est["recall_est"]
    st_p["recall_sample_rows"] = st_est["recall_sample_rows"]
    st_p["recall_sample_matches"] = st_est["recall_sample_matches"]
    res_f, ms_plain = timed(lambda: pkg.ejoin_threshold(ctx, X, X, w.eps), 1, 1)
    n_plain = res_f.count
    st_f = pkg.ejoin_last_stats(ctx)
    fi, fj = res_f.i.cpu().numpy().view(np.uint32), res_f.j.cpu().numpy().view(np.uint32)
    keep = np.isin(fi, rows)
    plain_sample = set(zip(fi[keep].tolist(), fj[keep].tolist()))
    del res_f
    sample = {"rows": 16, "plain_pairs": len(plain_sample), "pruned_subset_of_plain": pruned_sample <= plain_sample,
              "pruned_recall_on_rows": len(pruned_sample & plain_sample) / max(1, len(plain_sample))}
    # the plain FP32 CUDA-core path on the first 65,536 rows against all rows (pairs/s extrapolated)
    with pkg.Ctx(device=0, prec="f32", flags=pkg.EJOIN_FLAG_TIMING) as cf:
        Xs = X[:65536]
        pkg.ejoin_threshold(cf, Xs, X, w.eps)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        pkg.ejoin_threshold(cf, Xs, X, w.eps)
        z.record()
        z.synchronize()
        f32_pps = Xs.shape[0] * X.shape[0] / (a.elapsed_time(z) * 1e-3)
    logical = X.shape[0] * X.shape[0]
    out = {"metric": METRIC, "value": logical / (ms_pruned * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": max(2, args.steps), "warmup": max(3, args.warmup), "ms_per_step": round(ms_pruned, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": w.name + ", learned tile pruning (768-256-64 GELU sketch)",
                      "pairs_per_step": logical, "eps_sketch": eps_sk, "train_pairs": 10_000_000,
                      "training": train_rep},
           "pruned": st_p, "plain_bf16": {"ms_per_step": round(ms_plain, 2), "pairs": int(n_plain),
                                          "ms_contract": st_f["ms_contract"], "ms_rescore": st_f["ms_rescore"]},
           "recall": n_pruned / max(1, n_plain), "speedup_vs_plain_bf16": ms_plain / ms_pruned,
           "plain_fp32_cuda_cores": {"pairs_per_s": f32_pps, "sample": "first 65,536 rows x all rows"},
           "speedup_vs_plain_fp32": (logical / (ms_pruned * 1e-3)) / f32_pps,
           "gpu_launches": None, "sampled_rows": sample}
    if emit:
        print(json.dumps(out), flush=True)
    sk.close()
    ctx.close()
    del X, Xtr, Xcal
    torch.cuda.empty_cache()
    return out


def measure_library_peaks():
    """cuBLAS dense throughput on this GPU for the three tensor-core input types of the contraction
    (8192^3 products, 50 timed iterations after 5 warm-up ones): context for the nominal FP8/BF16 and
    TF32/BF16 ratios the rooflines use."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = True
    n = 8192

    def timeit(fn, iters=50):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(iters):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / iters

    out = {}
    A = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    B = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    out["bf16_tflops"] = 2 * n ** 3 / timeit(lambda: A @ B) / 1e9
    A32, B32 = A.float(), B.float()
    out["tf32_tflops"] = 2 * n ** 3 / timeit(lambda: A32 @ B32) / 1e9
    A8 = A.to(torch.float8_e4m3fn)
    B8 = B.to(torch.float8_e4m3fn).t().contiguous().t()
    one = torch.ones((), device="cuda")
    out["fp8_e4m3_tflops"] = 2 * n ** 3 / timeit(
        lambda: torch._scaled_mm(A8, B8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)) / 1e9
    out["tf32_over_bf16"] = out["tf32_tflops"] / out["bf16_tflops"]
    out["fp8_over_bf16"] = out["fp8_e4m3_tflops"] / out["bf16_tflops"]
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ejoin", choices=["ejoin", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp8", "tf32", "f32"])
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "c2-capture", "c1", "c3", "c3-capture", "c4", "c5", "top1", "top1-capture",
                             "top32", "top32-capture", "esel"])
    ap.add_argument("--esel-rows", type=int, default=10_000_000, help="rows of R for --workload esel")
    ap.add_argument("--c5-rows", type=int, default=4_000_000,
                    help="rows of --workload c5 (4,000,000: the configuration; fewer: a small case of the same shape)")
    ap.add_argument("--batch-jobs", type=int, default=512,
                    help="jobs of --workload c4 (512: the configuration; fewer: a small case of the same shape)")
    ap.add_argument("--peaks", action="store_true", help="print cuBLAS BF16 / TF32 / FP8 throughput and exit")
    ap.add_argument("--sel-pct", type=int, default=100,
                    help="top-k workloads: percent of S kept by the predicate attr < sel-pct")
    ap.add_argument("--cpu-s", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-step-s", type=float, default=4.0, help="seconds of oracle work per reference step")
    ap.add_argument("--group-m", type=int, default=0, help="contraction raster group width (0: auto)")
    ap.add_argument("--gather-rescore", action="store_true",
                    help="re-score in emission order (EJOIN_FLAG_GATHER_RESCORE) instead of by panels of R rows")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large-join", action="store_true",
                    help="skip the 2M-row self-join (large_join) the default line adds after the c2 workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched (c4) and learned (c5) summaries the default line adds after the c2 workload")
    ap.add_argument("--no-parity", action="store_true", help="accepted for compatibility; parity lives in tests/")
    args = ap.parse_args()
    if args.peaks:
        measure_library_peaks()
        return
    if args.warmup < 3 and args.impl == "ejoin":
        log("warning: fewer than 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4":
        run_batch(args)
    elif args.workload == "c5":
        run_learned(args)
    elif args.workload.startswith("top"):
        run_topk(args)
    elif args.workload == "esel":
        run_eselect(args)
    else:
        run_ejoin(args)


if __name__ == "__main__":
    main()
