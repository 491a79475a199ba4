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
    # the config names the sample this arm evaluates per step (not the GPU arm's 84M tuples)
    assert line["config"]["fact_tuples"] == 5000 and "5000 fact tuples" in line["config"]["workload"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_traffic_is_taken_only_from_a_capture_of_the_same_kernel(tmp_path, monkeypatch):
    """roofline.traffic comes from a committed ncu capture of the exact generated kernel (the
    hash of its source text), scaled by tuples; any other kernel gets no traffic figure."""
    import bench
    os.makedirs(tmp_path / "profiles")
    rec = [{"kernel": "lmfao_gen_root_pass", "source_hash": "abc", "tuples": 40_000_000, "read": 366_000_000,
            "write": 34_000_000, "bytes_per_tuple": 8}]
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    t40, src = bench.measured_traffic(40_000_000, {"generated": True, "source_hash": "abc"})
    t84, _ = bench.measured_traffic(84_000_000, {"generated": True, "source_hash": "abc"})
    assert t40 == 400_000_000 and t84 - t40 == 44_000_000 * 8 and "scaled" in src
    t, why = bench.measured_traffic(84_000_000, {"generated": True, "source_hash": "other"})
    assert t is None and "changed" in why
    assert bench.measured_traffic(84_000_000, {"generated": False})[0] is None


def test_parity_report_flags_errors_per_family():
    """The bench's parity summary: exact counts, per-family relative error against the sum of
    absolute terms, and a planted error in one aggregate shows up in its family only."""
    import numpy as np
    import bench
    from oracle import lmfao_oracle as O
    from paper_2008_08657_b300 import workloads as W
    rels = W.star_schema(n_fact=3000, seed=1)
    qs = W.star_batch()
    ref = O.evaluate(rels, qs)
    got = [{k: v.copy() for k, v in r.items()} for r in ref]
    rep = bench.parity_report(qs, got, ref, 1.0, 2, 1)
    assert rep["within_tolerance"] and rep["counts_exact"] and rep["max_rel_err"] == 0.0
    j = next(j for j, a in enumerate(qs[0]["aggs"]) if len(a) == 2)
    got[0]["sums"][0, j] += 1e-3 * ref[0]["abs"][0, j]
    rep = bench.parity_report(qs, got, ref, 1.0, 2, 1)
    assert not rep["within_tolerance"]
    fam = bench._family(qs[0], qs[0]["aggs"][j])
    assert abs(rep["families"][fam]["max_rel_err"] - 1e-3) < 1e-9
    assert all(f["max_rel_err"] == 0.0 for n, f in rep["families"].items() if n != fam)
    got[0]["counts"][0] += 1
    assert not bench.parity_report(qs, got, ref, 1.0, 2, 1)["counts_exact"]
