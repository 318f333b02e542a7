"""bench.py's roofline bookkeeping, on the CPU: the algorithmic bytes per launch, and the DRAM traffic taken
from the committed ncu record only while the kernel sources are the ones it was captured from."""
import json
import os

import pytest

import bench
from paper_1401_4350_gb300 import binding as B

KERNEL = "k_vertex_step_mixed<1,true>"


def _record():
    with open(os.path.join(bench.ROOT, "profiles", "dram_traffic.json")) as f:
        return json.load(f)[KERNEL]


def test_fused_algorithmic_bytes():
    # 4 B per list entry; 180 B per particle; 16 B more per particle over the inner list
    assert bench.algorithmic_bytes_fused(1000, 50000) == 4 * 50000 + 180 * 1000
    assert bench.algorithmic_bytes_fused(1000, 50000, inner=True) == 4 * 50000 + 196 * 1000
    assert bench.algorithmic_bytes_fused(0, 0) == 0


def test_force_algorithmic_bytes():
    # vertex: 4 B per entry + count 4 + own coordinates (16 mixed, 32 FP64) + force and virial 40
    assert bench.algorithmic_bytes_force(B.MD_VERTEX, B.MD_MIXED, 10, 300, 150) == 4 * 300 + 10 * 60
    assert bench.algorithmic_bytes_force(B.MD_VERTEX, B.MD_FP64, 10, 300, 150) == 4 * 300 + 10 * 76
    # edge: partner j 4 B per pair, row offsets, coordinates, outputs zeroed and accumulated once
    assert bench.algorithmic_bytes_force(B.MD_EDGE, B.MD_MIXED, 10, 300, 150) == 4 * 150 + 8 * 11 + 10 * (16 + 64)


def test_traffic_is_the_capture_at_its_own_size(monkeypatch):
    rec = _record()
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: rec["source_sha256"])
    t = bench.measured_traffic(KERNEL, rec["n"], rec["list_entries"])
    assert t == pytest.approx(rec["dram_bytes_per_launch"], rel=1e-12)
    assert rec["dram_bytes_per_launch"] == rec["dram_read"] + rec["dram_write"]


def test_traffic_scales_with_the_launch(monkeypatch):
    rec = _record()
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: rec["source_sha256"])
    t2 = bench.measured_traffic(KERNEL, 2 * rec["n"], 2 * rec["list_entries"])
    assert t2 == pytest.approx(2 * rec["dram_bytes_per_launch"], rel=1e-12)


def test_traffic_is_withheld_for_other_sources(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0" * 64)
    assert bench.measured_traffic(KERNEL, 1 << 20, 60_000_000) is None
    assert bench.measured_traffic("no_such_kernel", 1 << 20, 60_000_000) is None


def test_digest_covers_the_step_kernel_sources():
    d = bench.kernel_source_digest()
    assert len(d) == 64 and int(d, 16) >= 0


def test_fp64_peak_from_unit_counts():
    # 2 FP64 operations per clock per SM on 152 SMs: 629.28 G op/s at 2070 MHz
    assert bench.fp64_peak_gops(2070.0) == pytest.approx(2.0 * 152 * 2.070, rel=1e-12)
    assert bench.FP64_OPS_PER_PAIR_EVAL_LJ == 32
