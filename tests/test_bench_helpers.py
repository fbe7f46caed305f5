"""Host-side helpers of the benchmark (CPU): the roofline object of each
kernel kind from profiled statistics, and the hash guard of the recorded ncu
DRAM traffic."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Db:
    M, n, m = 10_000, 1_000_000, 1_000


def _stats(**kw):
    s = dict(count_ms=2.0, count_launches=100, count_ops=16 * 10**9, count_ops_timed=10**9,
             gram_ms=1.0, gram_launches=50,
             gram_flops=10**12, settle_ms=0.5, gen_ms=1.5, gen_launches=100,
             words_compact=16, l1=999, path_launches=[0, 0, 100, 50])
    s.update(kw)
    return s


def test_roofline_count_kind_is_alu_against_the_derived_peak():
    r = bench.roofline_of("count", [_stats()], {"count": 2.0}, 10.0, _Db())
    assert r["bound"] == "alu" and r["unit"] == "Top/s"
    # only the timed launches' work counts: 1e9 ops per 100 launches over 2
    # ms -> 1e7 ops per 20 us = 0.5 Top/s (the mine's 1.6e10 would overstate it)
    assert abs(r["achieved"] - 0.5) < 1e-9
    assert abs(r["frac"] - 0.5 / bench.ALU_PEAK_TOPS) < 1e-12


def test_roofline_count_kernel_follows_the_stop_loop_form():
    # per stop throughout, or handed over to the event-driven form (only the
    # per-stop stops are timed): the per-stop count kernel; event-driven
    # throughout: the cohort pass
    for loop, kern in ((0, "k_count_direct"), (2, "k_count_direct"), (1, "k_cohort_pass")):
        st = _stats(event_loop=loop, event_iters=3)
        r = bench.roofline_of("count", [st], {"count": 2.0}, 10.0, _Db())
        assert r["kernel"] == kern, (loop, r["kernel"])
        assert ("loop iteration" in r["timed_stops"]) == (loop == 1)
        assert ("per-stop part" in r["timed_stops"]) == (loop == 2)


def test_roofline_gram_kind_is_tensor_against_fp8_peak():
    r = bench.roofline_of("gram", [_stats()], {"gram": 1.0}, 10.0, _Db())
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    # 1e12 flops over 50 launches in 1 ms -> 2e10 per 20 us = 1000 TFLOP/s
    assert abs(r["achieved"] - 1000.0) < 1e-6
    assert r["peak"] == bench.peaks()["bf16"] * bench.FP8_PER_BF16


def test_roofline_gen_kind_counts_bytes_from_the_trace():
    trace = np.zeros((4, 9), dtype=np.uint64)
    trace[:, 5] = [10, 0, 0, 0]   # promoted
    trace[:, 7] = [0, 2, 0, 0]    # generated
    r = bench.roofline_of("gen", [_stats()], {"gen": 1.5}, 10.0, _Db(), trace=trace)
    want = (10 * 999 * 2 + 2 * (16 * 8 + 32 + 10)) / 4
    assert r["bound"] == "hbm" and abs(r["bytes_per_launch"] - want) < 1e-9


def test_traffic_guard_follows_the_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    import hashlib
    rec = {"k_x": {"dram_bytes_per_launch": 123.0, "sources": [str(src)],
                   "sources_sha256": hashlib.sha256(src.read_bytes()).hexdigest()}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    monkeypatch.setattr(bench, "ROOT", "/")
    assert bench.ncu_traffic("k_x") == 123.0
    assert bench.ncu_traffic("k_missing") is None
    src.write_text("kernel source, changed\n")
    assert bench.ncu_traffic("k_x") is None


def test_committed_traffic_record_names_existing_sources():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    assert {"k_count_direct", "k_generate_finish", "k_gram_pairs"} <= set(rec)
    for entry in rec.values():
        assert entry["dram_bytes_per_launch"] > 0
        for rel in entry["sources"]:
            assert os.path.exists(os.path.join(ROOT, rel))
