"""bench.py --impl reference, on the CPU: the FP64 oracle timed as it stands after the requested warm-up steps,
and the JSON line the benchmark contract asks for (metric, unit and direction of our arm, the timed steps,
a cpu_baseline and an e2e object that describe this run).  The workload is shrunk here to LJ N = 4000 so
that the test takes seconds; the arithmetic path is the one the bench runs."""
import argparse

import bench
from paper_1401_4350_gb300 import systems


def test_reference_arm_line(monkeypatch):
    monkeypatch.setattr(bench, "make_system", lambda rank=0: systems.make_lj(4000, 0.85, 1.0, seed=1001))
    line = bench.run_reference(argparse.Namespace(steps=4, warmup=3, gpus=1))
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "steps/s" and line["higher_is_better"] is True
    assert line["steps"] == 4 and line["requested_steps"] == 4 and line["warmup"] == 3
    assert line["value"] > 0 and abs(line["ms_per_step"] - 1e3 / line["value"]) < 1e-6 * line["ms_per_step"]
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and "3 warm-up" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
