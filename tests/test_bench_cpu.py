"""Host-side pieces of bench.py (no GPU): the roofline denominators and the DRAM
traffic it reports only for the kernel sources the committed ncu counters were
taken on."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_peaks_come_from_the_measured_file(bench):
    peak, source = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert source == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert source == "fallback" and peak == bench.FALLBACK_HBM_GBS


def test_source_hashes_follow_each_kernels_files(bench):
    # the two tile kernels share their sources; the prologue has its own
    assert bench.source_hash("k_compress") == bench.source_hash("k_decompress")
    assert bench.source_hash("k_compress") != bench.source_hash("k_prologue")
    assert len(bench.source_hash("k_compress")) == 16


def test_traffic_only_for_matching_sources(bench, tmp_path, monkeypatch):
    committed = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    for k in ("k_compress", "k_decompress"):
        entry = committed["kernels"][k]
        want = entry["dram_bytes_per_launch_full_size"] if entry["source_hash"] == bench.source_hash(k) else None
        assert bench.ncu_traffic(k) == want
    # a stale hash reads as no traffic at all
    stale = json.loads(json.dumps(committed))
    stale["kernels"]["k_compress"]["source_hash"] = "0" * 16
    fake_root = tmp_path / "repo"
    (fake_root / "profiles").mkdir(parents=True)
    (fake_root / "profiles" / "ncu_traffic.json").write_text(json.dumps(stale))
    (fake_root / "paper_2312_05492_gb300").symlink_to(os.path.join(ROOT, "paper_2312_05492_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    assert bench.ncu_traffic("k_compress") is None
    assert bench.ncu_traffic("not_a_kernel") is None
