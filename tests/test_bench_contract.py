"""bench.py on the CPU: the reference arm's JSON line (the oracle on a bounded sample) has the
keys of the contract, and the DRAM traffic of the root pass is read from the committed ncu
summary and scaled to the fact size."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-rows", "5000"], capture_output=True, text=True, check=True,
                         cwd=ROOT, timeout=600).stdout
    line = json.loads(out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["fact_tuples"] == 84_000_000  # the GPU arm's workload; the sample is in cpu_baseline
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_traffic_from_the_committed_capture_scales_with_tuples():
    import bench
    t40, src = bench.measured_traffic("retailer", 40_000_000, {"generated": True})
    t84, _ = bench.measured_traffic("retailer", 84_000_000, {"generated": True})
    assert src and t40 > 40_000_000 * 8 and t84 - t40 == 44_000_000 * 8
    assert bench.measured_traffic("retailer", 84_000_000, {"generated": False}) == (None, None)
    assert bench.measured_traffic("favorita", 84_000_000, {"generated": True}) == (None, None)
