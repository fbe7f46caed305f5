#!/usr/bin/env python
"""Benchmark: candidate-transaction tests/s and DIC mine time on one GB300.

A step is one complete mining call (first pass, pair join and every stop of
Algorithm 2's loop until DASHED is empty, result on the host) over the
paper-scale planted-pattern database (n=1,000,000 rows, m=1,000 items,
minsup 0.25% = 2,500, M=10,000), resident in HBM when the timed region starts.
The L2 cache is flushed (a 512 MiB write) before every timed step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The count configuration is the autotuner's choice for the query (timed on it,
every candidate checked to give the same result); `--path` forces one,
`--no-tune` keeps the library's rule, `--algorithm classic` runs Algorithm 1.
Other workloads: `--workload dense|batched|served|planted-small`; `--sweep`
times both algorithms over block sizes and thresholds (one JSON line).

`--impl reference` times the CPU oracle (the plain serial restatement of the
paper's algorithm) on the host cores instead, on a bounded sample of the same
workload. With N > 1 (torchrun) every rank mines its own replica; the value is
the sum of tests over all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "candidate-transaction tests/s (DIC mine, bit-exact)"
UNIT = "tests/s"
# One sample of the oracle for the CPU figures: the first pass over all rows
# plus the first stop of all pair candidates over a block of this many rows.
CPU_SAMPLE_M = 1_000

# Derived integer-ALU peak: 152 SMs x 64 INT32 lanes x 2070 MHz (max SM
# clock). The count kernels report their algorithmic integer work (ROWS: one
# LOP3 per touched 32-bit half + compare + add per test; BITSLICE: k-1 AND +
# POPC + ADD per 32-row word) in stats["count_ops"].
ALU_PEAK_TOPS = 152 * 64 * 2.070e9 / 1e12
COUNT_KERNELS = {1: "k_count_rows", 2: "k_count_direct", 3: "k_count_direct"}  # (k_count_bitslice for large windows)
# fp8 (kind::f8f6f4) dense tensor peak = the measured bf16 peak x 2, the
# nominal fp8:bf16 ratio (4.5 / 2.25 PFLOP/s)
FP8_PER_BF16 = 2.0
# the timed steps bracket the dominant kernel kind with CUDA events on one
# stop in this many
PROFILE_EVERY = 64
# timed kinds of the stop loop: stats key prefix -> profile name, kernels
KINDS = {"count": "count", "gram": "gram", "settle": "settle", "gen": "gen"}
KIND_KERNELS = {"gram": "k_gram_pairs", "settle": "k_settle_pairs",
                "gen": "k_generate_finish"}


def workload(name: str):
    if name == "paper-scale":
        return synth.planted_paper_scale()
    if name == "planted-small":
        return synth.planted_small()
    if name == "dense":
        return synth.dense_zipf()
    raise SystemExit(f"unknown workload {name}")


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or
    None when there is none or a source file it was built from has changed
    since (the file records their SHA-256)."""
    import hashlib
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        entry = json.load(f).get(kernel)
    if not entry:
        return None
    h = hashlib.sha256()
    for rel in entry["sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return entry["dram_bytes_per_launch"] if h.hexdigest() == entry["sources_sha256"] else None


def roofline_of(kind, stats, shares_ms, step_ms, db, count_form="auto", trace=None,
                alu_peak=None):
    """Roofline object of the kernel kind `kind` from the profiled timed steps."""
    pk = peaks()
    tot_ms = sum(s[kind + "_ms"] for s in stats)
    nkey = {"count": "count_launches", "gram": "gram_launches", "gen": "gen_launches"}
    # one PRUNE-of-pairs launch per tensor-counted stop
    nl = sum(s[nkey[kind]] if kind in nkey else s["path_launches"][3] for s in stats)
    avg_ms = tot_ms / max(nl, 1)
    st = stats[0]
    # event_loop 1: event-driven throughout; 2: per stop, then handed over
    # (only the per-stop stops are timed)
    ev = st.get("event_loop") == 1
    common = {"avg_launch_ms": avg_ms, "launches_timed": nl,
              "timed_stops": (f"one loop iteration in {PROFILE_EVERY} of the timed steps" if ev
                              else f"one stop in {PROFILE_EVERY} of the per-stop part of the "
                              "timed steps" if st.get("event_loop") == 2
                              else f"one stop in {PROFILE_EVERY} of the timed steps"),
              "kind_ms_per_step_warmup": {k: v for k, v in shares_ms.items()}}
    if kind == "gram":
        flops = sum(s["gram_flops"] for s in stats) / max(nl, 1)
        ach = flops / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0
        peak = pk["bf16"] * FP8_PER_BF16
        return dict(bound="tensor", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    traffic=ncu_traffic(KIND_KERNELS[kind]), kernel=KIND_KERNELS[kind],
                    peak_source=f"{pk['source']} bf16 burst x {FP8_PER_BF16} (fp8 e4m3)",
                    flops_per_launch=flops, **common)
    if kind == "count":
        # work of the launches the events bracketed (the stops whose count
        # kernel was timed), per launch
        ops = sum(s["count_ops_timed"] for s in stats) / max(nl, 1)
        ach = ops / (avg_ms / 1e3) / 1e12 if avg_ms > 0 else 0.0
        pl = st["path_launches"]
        kern = COUNT_KERNELS[max((1, 2, 3), key=lambda i: pl[i])]
        if kern != "k_count_rows" and count_form == "tiled":
            kern = "k_count_bitslice"
        if ev:  # the event-driven loop counts each cohort over its whole pass
            kern = "k_cohort_pass"
        peak = alu_peak if alu_peak else ALU_PEAK_TOPS
        src = ("measured in this run: lop3.b32 issue rate (dic_measure_alu_peak)" if alu_peak
               else "derived: 152 SM x 64 INT32 lanes x 2070 MHz")
        return dict(bound="alu", achieved=ach, peak=peak, unit="Top/s", frac=ach / peak,
                    traffic=ncu_traffic(kern), kernel=kern, peak_source=src,
                    derived_peak=ALU_PEAK_TOPS, ops_per_launch=ops, **common)
    # gen / settle: latency-bound memory-side kernels; algorithmic bytes per launch
    wc, l1 = st["words_compact"], st["l1"]
    if kind == "gen":
        # MAKECANDIDATES + CHECKFULLPASS (the next block's transposition runs
        # beside the count): per (promoted record, rank) two pair-record
        # shape bytes read, per emitted candidate its record written (mask
        # W'*8 + ranks 32 + count, birth, shape, size 10 bytes), from the trace
        if trace is not None and len(trace):
            promoted, generated = float(trace[:, 5].sum()), float(trace[:, 7].sum())
            # one launch per stop, or per loop iteration (event-driven loop)
            nlaunch = st["event_iters"] if ev and st.get("event_iters") else len(trace)
            byts = (promoted * l1 * 2 + generated * (wc * 8 + 32 + 10)) / nlaunch
        else:
            byts = 0.0
    else:
        # every pair record's counter, shape and birth read once
        byts = l1 * (l1 - 1) / 2 * 9
    ach = byts / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
    return dict(bound="hbm", achieved=ach, peak=pk["hbm_gbs"], unit="GB/s",
                frac=ach / pk["hbm_gbs"], traffic=ncu_traffic(KIND_KERNELS[kind]),
                kernel=KIND_KERNELS[kind],
                peak_source=f"{pk['source']} copy bandwidth", bytes_per_launch=byts, **common)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=d.get("hbm_gbs", 6800.0), bf16=d.get("bf16_tflops", 1900.0),
                    bf16_sus=d.get("bf16_tflops_sustained", 1700.0), source="measured")
    return dict(hbm_gbs=6800.0, bf16=1900.0, bf16_sus=1700.0, source="fallback")


class Clocks:
    """nvidia-smi sampling every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        with open(self.f.name) as f:
            lines = [ln.strip() for ln in f if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_sample(db):
    """Time the oracle on the bounded sample; returns (tests/s, tests, seconds)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, CPU_SAMPLE_M, max_stops=1)
    dt = time.perf_counter() - t0
    return r.tests / dt, r.tests, dt


def cpu_sample_desc(db):
    return (f"oracle (serial C++ ParallelDIC) on the same database: first pass over all "
            f"{db.n} rows + the first stop of all pair candidates over a {CPU_SAMPLE_M}-row "
            f"block (M={CPU_SAMPLE_M} instead of {db.M} to bound the sample)")


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# The multi-core baseline's sample of the paper-scale workload: the first
# pass over all rows and the first stops of the loop at the workload's own M.
PDIC_SAMPLE_STOPS = 2


def cpu_paralleldic(db):
    """The paper's own parallel design (ParallelDIC with OpenMP, Algorithms
    2-5 with the loop interchange and nested balancing of Figures 2-3) on
    every host core: the complete planted-small mine (its result checked
    against the serial oracle) and a bounded sample of `db`."""
    import oracle
    small = synth.planted_small()
    t0 = time.perf_counter()
    r1, used = oracle.paralleldic(small.row_ptr, small.items, small.n, small.m, small.minsup,
                                  small.M)
    c1_s = time.perf_counter() - t0
    ref = oracle.dic(small.row_ptr, small.items, small.n, small.m, small.minsup, small.M,
                     superset_loop=False)
    same = r1.itemsets == ref.itemsets and r1.trace.tolist() == ref.trace.tolist()
    t0 = time.perf_counter()
    r2, _ = oracle.paralleldic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M,
                               max_stops=PDIC_SAMPLE_STOPS)
    dt = time.perf_counter() - t0
    return {"value": r2.tests / dt, "unit": UNIT, "cores": used, "cpu_model": cpu_model(),
            "nproc": os.cpu_count(), "kind": "ParallelDIC, OpenMP (the paper's design)",
            "sample": (f"{db.name}: first pass over all {db.n} rows + the first "
                       f"{PDIC_SAMPLE_STOPS} stops at M={db.M} ({r2.tests} tests in {dt:.1f} s)"),
            "planted_small_full_mine_ms": 1000 * c1_s,
            "planted_small_tests_per_s": r1.tests / c1_s,
            "planted_small_equal_to_oracle": bool(same)}


def aggregate_replicas(seconds: float, tests: float, device: str):
    """Whole-job figures over the replicas (one process per GPU, each mining
    its own copy): the slowest rank's time and the sum of the ranks' tests.
    Without an initialised process group of more than one rank, the inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds, float(tests)
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    n = torch.tensor([float(tests)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t[0]), float(n[0])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    db = workload(args.workload)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        cpu_sample(db)
    tests, secs = 0, 0.0
    for _ in range(args.steps):
        _, t, dt = cpu_sample(db)
        tests += t
        secs += dt
    v = tests / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": db.name, "n": db.n, "m": db.m,
                                        "minsup": db.minsup, "M": db.M,
                                        "sample": cpu_sample_desc(db)},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": cpu_sample_desc(db)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args, dic, torch):
    """Mine time of both algorithms over block sizes M and support thresholds
    on one database (the analogue of the paper's study of M): every point
    is checked to give the same itemsets under both algorithms."""
    db = workload(args.workload)
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    points = []
    for frac in (0.0025, 0.005, 0.01):
        minsup = synth.minsup_count(db.n, frac)
        for M in sorted({db.n // 400, db.n // 100, db.n // 20, db.n // 2}):
            row = {"minsup": minsup, "M": M}
            ref = None
            for alg in ("paralleldic", "classic"):
                for _ in range(args.warmup):
                    r = dic.mine(h, minsup, M, algorithm=alg)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(args.steps):
                    r = dic.mine(h, minsup, M, algorithm=alg)
                dt = (time.perf_counter() - t0) / args.steps
                sig = r.itemsets()
                assert ref is None or sig == ref, "algorithms disagree"
                ref = sig
                row[alg] = {"ms": 1000 * dt, "tests": int(r.stats["tests"]),
                            "stops": int(r.stats["stops"]), "tests_per_s": r.stats["tests"] / dt}
            row["frequent_itemsets"] = len(ref)
            points.append(row)
    print(json.dumps({"sweep": "mine time over M and minsup (wall clock, result on the host)",
                      "workload": db.name, "steps": args.steps, "warmup": args.warmup,
                      "points": points}), flush=True)
    return 0


def run_batched(args, dic, torch):
    """512 databases of the batched recipe mined together (one dic_mine_batch
    per step), against plain per-query GPU DIC (ROWS path, one query at a
    time) and against the single-query fast path run query by query."""
    n_db = args.batch_dbs
    dbs = [synth.batched_db(i) for i in range(n_db)]
    hs = [dic.load_db_csr(d.row_ptr, d.items, d.n, d.m) for d in dbs]
    ms = [d.minsup for d in dbs]
    Ms = [d.M for d in dbs]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn, steps):
        out, t = None, 0.0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
        return out, t / steps

    # the tile width common to the batch's rounds, timed on the batch itself
    from paper_1812_10959_gb300 import autotune
    tuned = autotune.Tuner(repeats=1).tune_batch(hs, ms, Ms)
    tw = tuned.tile_words
    for _ in range(args.warmup):
        res = dic.mine_batch(hs, ms, Ms, tile_words=tw)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    res, t_batch = timed(lambda: dic.mine_batch(hs, ms, Ms, tile_words=tw), args.steps)
    clk = clocks.stop()
    tests = sum(r.stats["tests"] for r in res)
    single, t_single = timed(lambda: [dic.mine(h, m_, M_) for h, m_, M_ in zip(hs, ms, Ms)], 1)
    plain, t_plain = timed(lambda: dic.mine_batch(hs, ms, Ms, path="rows"), 1)
    same = all(a.itemsets() == b.itemsets() == c.itemsets() for a, b, c in zip(res, single, plain))
    launches = sum(r.stats["kernel_launches"] for r in res)
    line = {
        "metric": METRIC, "value": tests / t_batch, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_batch,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": f"batched {n_db} planted-pattern databases",
                   "rows_total": int(sum(d.n for d in dbs)), "tests_per_step": tests,
                   "l2": "flushed (512 MiB write) per step"},
        "queries_per_s": n_db / t_batch,
        "single_query_fast_path": {"queries_per_s": n_db / t_single, "ms": 1000 * t_single},
        "plain_per_query_gpu_dic": {"queries_per_s": n_db / t_plain, "ms": 1000 * t_plain},
        "identical_results": bool(same),
        "autotune": {"tile_words": tw, "candidates_s": tuned.timings},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_served(args, dic, torch):
    """64 databases of the batched recipe + 2 paper-scale databases, all
    device-resident; 10,000 queries arriving as a Poisson process at 200 req/s
    (database uniform, minsup log-uniform 0.2%-5%, M in {n/20, n/10, n/4}),
    served with continuous batching under a 120 GB HBM budget. Reports
    p50/p99 latency and queries/s, the server's capacity (all queries
    submitted at once), and plain per-query GPU DIC on a sample."""
    import threading
    raw = [synth.batched_db(i, base_seed=5000) for i in range(64)]
    raw += [synth.planted_paper_scale(seed=6000), synth.planted_paper_scale(seed=6001)]
    hs = [dic.load_db_csr(d.row_ptr, d.items, d.n, d.m) for d in raw]
    qs = []
    for q in synth.served_queries(args.served_queries, len(raw)):
        d = raw[q["db"]]
        qs.append((q["t"], q["db"], synth.minsup_count(d.n, q["frac"]), max(1, d.n // q["mdiv"])))
    budget, slots = 120 << 30, 64

    def serve(open_loop: bool):
        srv = dic.Server(budget, slots)
        tickets = [None] * len(qs)
        ready = threading.Semaphore(0)

        def submitter():
            t0 = time.perf_counter()
            for i, (t, db, ms, M) in enumerate(qs):
                if open_loop:
                    dt = t0 + t - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                tickets[i] = srv.submit(hs[db], ms, M)
                ready.release()

        th = threading.Thread(target=submitter)
        t_start = time.perf_counter()
        th.start()
        out = []
        for i in range(len(qs)):
            ready.acquire()
            out.append(srv.wait(tickets[i]))
        th.join()
        elapsed = time.perf_counter() - t_start
        st = srv.stats()
        srv.close()
        return out, st, elapsed

    serve(False) if args.warmup else None
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    res, st, el = serve(True)
    clk = clocks.stop()
    _, st_cap, el_cap = serve(False)
    k = min(args.plain_sample, len(qs))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [dic.mine(hs[db], ms, M, path="rows") for _, db, ms, M in qs[:k]]
    t_plain = time.perf_counter() - t0
    # the single-query fast path, one query after another, on the same sample
    t0 = time.perf_counter()
    fast = [dic.mine(hs[db], ms, M) for _, db, ms, M in qs[:k]]
    t_fast = time.perf_counter() - t0
    same = all(a.itemsets() == b.itemsets() == c.itemsets()
               for a, b, c in zip(res[:k], plain, fast))
    tests = sum(r.stats["tests"] for r in res)
    line = {
        "metric": METRIC, "value": tests / el, "unit": UNIT, "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": 1000 * el, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "served: 64 batched-recipe + 2 paper-scale databases, "
                               f"{len(qs)} Poisson arrivals at 200 req/s",
                   "hbm_budget_gb": 120, "slots": slots},
        "served": {"queries_per_s": st["qps"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                   "mean_ms": st["mean_ms"], "peak_slots": st["peak_slots"],
                   "rounds": st["rounds"], "elapsed_s": el},
        "capacity": {"queries_per_s": len(qs) / el_cap, "p50_ms": st_cap["p50_ms"],
                     "p99_ms": st_cap["p99_ms"], "peak_slots": st_cap["peak_slots"]},
        "plain_per_query_gpu_dic": {"queries_per_s": k / t_plain, "sample": k},
        "single_query_fast_path": {"queries_per_s": k / t_fast, "sample": k},
        "solo_queries": st["solo"],
        "identical_results_on_sample": bool(same),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper-scale")
    ap.add_argument("--path", default="auto", choices=["auto", "rows", "bitslice", "tensor"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline sample")
    ap.add_argument("--no-tune", action="store_true",
                    help="with --path auto: use the library's rule instead of the autotuner")
    ap.add_argument("--algorithm", default="paralleldic", choices=["paralleldic", "classic"],
                    help="classic: Algorithm 1 (no first pass; every item a dashed circle)")
    ap.add_argument("--sweep", action="store_true",
                    help="mine time over M and minsup for both algorithms (one JSON line)")
    ap.add_argument("--batch-dbs", type=int, default=512, help="databases for --workload batched")
    ap.add_argument("--served-queries", type=int, default=10_000)
    ap.add_argument("--plain-sample", type=int, default=300,
                    help="queries of the served stream timed with plain per-query GPU DIC")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1812_10959_gb300 import build as pb
    pb.build()
    import paper_1812_10959_gb300 as dic

    if args.sweep:
        return run_sweep(args, dic, torch)
    if args.workload == "batched":
        return run_batched(args, dic, torch)
    if args.workload == "served":
        return run_served(args, dic, torch)
    db = workload(args.workload)
    handle = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()

    # count configuration: the autotuner's choice for this query (timed on the
    # query itself, all candidates checked to give the same result), or the
    # path given on the command line
    tuned = None
    if args.algorithm != "paralleldic":
        kw = dict(path=args.path, algorithm=args.algorithm)
    elif args.path == "auto" and not args.no_tune:
        from paper_1812_10959_gb300 import autotune
        tuned = autotune.Tuner(repeats=2).tune(handle, db.minsup, db.M)
        kw = tuned.kwargs()
    else:
        kw = dict(path=args.path)
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            # the last warm-up step times every kernel kind of the stop loop
            res = dic.mine(handle, db.minsup, db.M, **kw, stream=stream,
                           profile=(i == args.warmup - 1))
    ref_count = len(res.k)
    shares_ms = {k: res.stats[k + "_ms"] for k in KINDS}
    kind = max(shares_ms, key=lambda k: shares_ms[k])
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    evs = []
    stats = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            # the dominant kernel kind is bracketed by events inside the step,
            # on one stop in PROFILE_EVERY (each timed stop adds two event
            # records to its graph)
            res = dic.mine(handle, db.minsup, db.M, **kw, stream=stream,
                           profile=[kind, "gram"], profile_every=PROFILE_EVERY)
            b.record(stream)
            evs.append((a, b))
            stats.append(res.stats)
            assert len(res.k) == ref_count
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    total_s = sum(ms) / 1000.0
    tests_step = stats[0]["tests"]
    tests_all = tests_step * args.steps
    t_max, tests_all = aggregate_replicas(total_s, tests_all, "cuda")
    value = tests_all / t_max

    # ---- end to end through the C ABI from host buffers: the rows as CSR
    # item lists in pinned host memory are copied in, packed on the device,
    # mined, and the result read back, every step
    rp_h = torch.from_numpy(db.row_ptr.view(np.int64)).pin_memory()
    it_h = torch.from_numpy(db.items.view(np.int32)).pin_memory()
    e2e_s = 0.0
    d2h = 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2 = dic.load_db_csr(rp_h, it_h, db.n, db.m)
        r2 = dic.mine(h2, db.minsup, db.M, **kw)
        h2.free()
        e2e_s += time.perf_counter() - t0
        d2h = r2.masks.nbytes + r2.k.nbytes + r2.support.nbytes + r2.trace.nbytes
    h2d = rp_h.numel() * 8 + it_h.numel() * 4
    e2e_max, e2e_tests = aggregate_replicas(e2e_s, tests_step * args.steps, "cuda")
    e2e_v = e2e_tests / e2e_max

    # ---- roofline of the dominant kernel kind, timed live with CUDA events
    # on the mining stream around each of its launches in the timed steps
    try:
        alu_peak = dic.dic.measure_alu_peak()
    except Exception:  # noqa: BLE001 (the derived peak is used instead)
        alu_peak = None
    roofline = roofline_of(kind, stats, shares_ms, sum(ms), db, kw.get("count_form", "auto"),
                           res.trace, alu_peak)
    # the pair-cohort GEMM (one launch per mine when the pass is staged) is
    # timed in every step as well
    roofline_gram = (roofline_of("gram", stats, shares_ms, sum(ms), db) if kind != "gram" and
                     sum(s["gram_launches"] for s in stats) else None)

    cpu = pdic = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, t, dt = cpu_sample(db)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": cpu_sample_desc(db) + f" ({t} tests in {dt:.1f} s)",
               "cpu_model": cpu_model()}
        pdic = cpu_paralleldic(db)

    launches = sum(s["kernel_launches"] for s in stats)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": db.name, "n": db.n, "m": db.m, "minsup": db.minsup,
                       "M": db.M, "algorithm": args.algorithm,
                       "count_path": (f"autotuned: {tuned.path}, tile_words {tuned.tile_words}, "
                                      f"count form {tuned.count_form}") if tuned else args.path,
                       "tests_per_step": tests_step,
                       "frequent_itemsets": ref_count, "l2": "flushed (512 MiB write) per step",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "roofline_gram": roofline_gram,
            "autotune": ({"choice": tuned.kwargs(), "candidates_s": tuned.timings}
                         if tuned else None),
            "cpu_baseline": cpu,
            "cpu_paralleldic": pdic,
            "clocks": clk,
            "stats": stats[0],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
