"""Throughput of one aggregate batch over a join: fact tuples/s on one B300.

Workload: the Retailer-shaped 5-relation snowflake (84M fact tuples; Item 3,700 x 4 features,
Location 1,300 x 10 -> Census 1,300 x 14, Weather 160,000 (locn, date) pairs x 8 features;
3 categoricals of 24/12/50 values) with its ridge-regression batch: COUNT, 37 SUM(x),
703 SUM(x_i x_j), one-hot group-bys per categorical and per categorical pair
(Section 3, linear regression). Seeded synthetic data of that shape stand in for the
Retailer dataset.

A step is one lmfao_run of the whole batch (view kernels, root pass, combine) with the
relations resident in HBM; the fact columns (1.3 GB) exceed L2, so no flush is needed.
Prints one JSON line (the driver's contract) with roofline, CPU-oracle baseline, clocks,
and an end-to-end number through the C ABI from pinned host buffers.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fact tuples/s per aggregate batch"
UNIT = "tuples/s"


def tensor_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1800.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


WORKLOADS = {
    "retailer": ("retailer-snowflake ridge batch", 84_000_000),
    "favorita": ("favorita-schema ridge + categorical-pair batch", 120_000_000),
    "star": ("star-join ridge batch", 200_000),
    "dt": ("decision-tree level (8 leaves x 37 features x 20 buckets) on the retailer snowflake", 84_000_000),
}


def workload(n_fact, seed=0, which="retailer"):
    from paper_2008_08657_b300 import workloads as W
    if which == "favorita":
        return W.favorita_schema(n_fact=n_fact, seed=seed), W.favorita_batch()
    if which == "star":
        return W.star_schema(n_fact=n_fact, seed=seed), W.star_batch()
    rels = W.retailer_schema(n_fact=n_fact, seed=seed)
    if which == "dt":
        return rels, W.dt_level_batch(rels, seed=seed)[0]
    return rels, W.retailer_batch()


def measured_traffic(n_fact, root_pass):
    """DRAM bytes per root-pass launch from the committed capture of the same generated kernel
    (profiles/traffic.json, keyed by the hash of the kernel's source text), scaled from the
    captured fact size to n_fact by the per-tuple column bytes (the per-segment parts do not
    change with the fact size). (None, reason) when no capture of this exact kernel exists."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not root_pass or not root_pass.get("generated"):
        return None, "root pass not generated"
    try:
        with open(path) as f:
            caps = json.load(f)
    except (OSError, ValueError):
        return None, "no committed capture"
    for c in caps:
        if c.get("kernel") == "lmfao_gen_root_pass" and c.get("source_hash") == root_pass.get("source_hash"):
            t = c["read"] + c["write"] + (n_fact - c["tuples"]) * c["bytes_per_tuple"]
            return t, f"ncu capture of this kernel at {c['tuples']} fact tuples (profiles/traffic.json), scaled by tuples"
    return None, "kernel changed since the last capture (no capture of this source hash)"


def workload_config(args, n_fact, qs):
    return {"workload": f"{WORKLOADS[args.workload][0]}, {n_fact} fact tuples, {len(qs)} queries, "
                        f"{sum(len(q['aggs']) for q in qs)} aggregates", "fact_tuples": n_fact}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self):
        self.path = tempfile.mktemp(suffix=".csv")
        self.p = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"),
                                       f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
            rows = [[x.strip() for x in r] for r in rows if len(r) >= 7]
            sm = [float(r[0]) for r in rows]
            mx = max(float(r[1]) for r in rows)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower().startswith("active")})
            return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}
        except Exception as e:  # noqa: BLE001
            return {"error": str(e)}


def time_runs(eng, torch, stream, steps, warmup, merge=None):
    """``merge`` (N > 1): the all-reduce of the ranks' result states, after each run on the
    same stream; it is part of the step."""
    def step():
        eng.run(stream)
        if merge is not None:
            with torch.cuda.stream(stream):
                merge()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    fact_ms = []
    evs[0].record(stream)
    for i in range(steps):
        step()
        evs[i + 1].record(stream)
        kt = None
        if eng._profiling:
            kt = eng.kernel_times()
            fact_ms.append(sum(ms for n, ms in kt if n == "fact_pass"))
    torch.cuda.synchronize()
    ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    return ms, fact_ms


def bench_lmfao(args):
    import torch
    from paper_2008_08657_b300.lmfao import Engine

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # weak scaling: every rank holds a full-size shard of the fact relation of its own (seeded
    # by rank) and the replicated dimensions; the ranks' result states are summed each step
    rels, qs = workload(args.fact_rows, seed=args.seed + rank, which=args.workload)
    n_fact = rels[0]["nrows"]
    eng = Engine(local)
    for R in rels:
        eng.load_relation(R)
    eng.add_queries(qs)
    info = eng.plan(precision=args.precision, autotune=args.autotune)
    desc = eng.describe()
    stream = torch.cuda.Stream()
    # kernel-level timing of the dominant kernel (CUDA events inside lmfao_run, same stream)
    eng.set_profiling(True)
    eng._profiling = True
    _, fact_ms = time_runs(eng, torch, stream, max(3, args.steps // 2), 2)
    kernel_ms = {}
    for name, ms_k in eng.kernel_times():
        kernel_ms[name] = round(ms_k, 4)
    eng.set_profiling(False)
    eng._profiling = False
    # the timed region proper
    merge = None
    if world > 1:
        from paper_2008_08657_b300.distributed import merge_state
        state = eng.result_state()
        merge = lambda: merge_state(*state)  # noqa: E731
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks() as clk:
        ms, _ = time_runs(eng, torch, stream, args.steps, args.warmup, merge)
    ms_step = float(np.mean(ms))
    if world > 1:
        t = torch.tensor([ms_step], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * n_fact / (ms_step / 1e3)
    # plain FP64 GPU form of the same plan shape (same batch, FP64 arithmetic)
    fp64_ms = None
    if not args.skip_fp64:
        eng64 = Engine(local)
        for R in rels:
            eng64.load_relation(R)
        eng64.add_queries(qs)
        eng64.plan(precision="fp64")
        eng64._profiling = False
        ms64, _ = time_runs(eng64, torch, stream, max(2, args.steps // 4), 1)
        fp64_ms = float(np.mean(ms64))
        eng64.close()
    # roofline of the dominant kernel
    peak, peak_kind = peaks()
    fbytes = desc["physical"]["fact_pass_bytes"]
    fms = float(np.mean(fact_ms)) if fact_ms else None
    achieved = fbytes / (fms / 1e3) / 1e9 if fms else None
    roofline = {"bound": "hbm", "kernel": "fact_pass", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "peak_source": peak_kind,
                "algorithmic_bytes": fbytes, "kernel_ms": fms, "traffic": None}
    traffic, tsrc = measured_traffic(n_fact, desc["physical"].get("root_pass"))
    roofline["traffic"] = traffic
    roofline["traffic_source"] = tsrc
    # the per-block contraction kernel of the combine, against HBM and against the tensor pipe
    comb = None
    czb, czf = desc["physical"].get("combine_z_bytes", 0), desc["physical"].get("combine_z_flops", 0)
    if czb and kernel_ms.get("combine_z"):
        t = kernel_ms["combine_z"] / 1e3
        comb = {"kernel": "combine_z", "contraction": desc["physical"].get("contraction"),
                "bound": "hbm", "algorithmic_bytes": czb, "achieved": czb / t / 1e9, "peak": peak, "unit": "GB/s",
                "frac": czb / t / 1e9 / peak, "flops": czf, "tflops": czf / t / 1e12,
                "kernel_ms": kernel_ms["combine_z"], "chunk": desc["physical"].get("combine_chunk")}
        if args.precision == "split_bf16":
            tp = tensor_peak()
            comb["tensor_frac"] = czf / t / 1e12 / tp if tp else None
            comb["tensor_peak_tflops"] = tp
    # end to end through the C ABI: pinned host -> device copies, load, plan, run, fetch
    got = eng.fetch_all() if rank == 0 and args.parity else None
    eng.close()
    e2e = None
    batches = None
    if not args.skip_e2e:
        e2e = bench_e2e(args, rels, qs, torch, local)
        batches = bench_batches(args, rels, qs, torch, local)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "split_bf16": "f32 (dense contraction as split bf16 x3)"}[args.precision],
        "data": f"synthetic (seeded, {args.workload}-shaped)",
        "config": {**workload_config(args, n_fact, qs), "precision": args.precision,
                   "l2": "inputs larger than L2 (no flush)",
                   "segments": info["n_segments"], "segment_relation": desc["physical"]["segment_relation"],
                   "parallelism": f"dp{world} (fact row shards; all-reduce of the result state each step)"
                   if world > 1 else "single GPU"},
        "roofline": roofline,
        "vs_plain_fp64_gpu": (fp64_ms / ms_step) if fp64_ms else None,
        "plain_fp64_ms_per_step": fp64_ms,
        "plan_ms": info["plan_ms"],
        "reorg_ms": info["reorg_ms"],
        "batches_from_resident_data": batches,
        "combine_roofline": comb,
        "tiles": desc["physical"].get("tiles"),
        "kernel_ms": kernel_ms,
        "root_pass_shape": dict(desc["physical"].get("root_pass") or {},
                                **{k: desc["physical"].get(k) for k in
                                   ("filter_family", "cta_items", "per_tuple_items", "segment_sums", "work_items")}),
        "combine_shape": {k: desc["physical"].get(k) for k in
                          ("block_combine", "projection_combine", "projection_entries", "combine_items",
                           "outer_terms",
                           "prefix_digits")},
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": info["n_kernels"] * args.steps,
    }
    if got is not None:
        # every aggregate against the oracle over the whole workload, on all host cores; the same
        # run is the CPU baseline
        par = full_parity(rels, qs, got)
        out["parity"] = par
        out["cpu_baseline"] = {"value": n_fact / par["oracle_s"], "unit": UNIT, "cores": par["oracle_cores"],
                               "kind": "oracle",
                               "sample": f"the whole workload ({n_fact} fact tuples, {par['oracle_chunks']} chunks "
                                         f"of 1M tuples over {par['oracle_cores']} processes), "
                                         f"{par['oracle_s']} s"}
    elif rank == 0 and not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def bench_e2e(args, rels, qs, torch, local):
    from paper_2008_08657_b300.lmfao import Engine
    pinned = []
    h2d = 0
    for R in rels:
        cols = []
        for c in R["columns"]:
            t = torch.from_numpy(np.ascontiguousarray(c["data"])).pin_memory()
            cols.append(t)
            h2d += t.numel() * t.element_size()
        pinned.append(cols)
    steps = max(2, args.steps // 5)
    times = []
    d2h = 0
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eng = Engine(local)
        for R, cols in zip(rels, pinned):
            dev = [c.cuda(non_blocking=True) for c in cols]
            torch.cuda.synchronize()
            eng.load_relation(dict(R, columns=[dict(c, data=d) for c, d in zip(R["columns"], dev)]), where="device")
        eng.add_queries(qs)
        eng.plan(precision=args.precision)
        eng.run()
        res = eng.fetch_all()
        t1 = time.perf_counter()
        eng.close()
        d2h = sum(r["counts"].nbytes + r["sums"].nbytes + r["keys"].nbytes for r in res)
        if i > 0:
            times.append(t1 - t0)
    s = float(np.mean(times))
    return {"value": rels[0]["nrows"] / s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "seconds_per_step": s,
            "includes": "pinned H2D of all relations, lmfao_load_relation, lmfao_plan (trie reorganisation), "
                        "lmfao_run, lmfao_fetch of every query"}


def bench_batches(args, rels, qs, torch, local):
    """Plan + run + fetch of a batch from relations already resident in HBM: the first batch on
    a new context (reorganises the root relation; the generated kernel is already compiled in
    this process) and a second batch on the same context (reuses the segment order)."""
    from paper_2008_08657_b300.lmfao import Engine
    dev = [[torch.from_numpy(np.ascontiguousarray(c["data"])).cuda() for c in R["columns"]] for R in rels]
    torch.cuda.synchronize()
    eng = Engine(local)
    for R, cols in zip(rels, dev):
        eng.load_relation(dict(R, columns=[dict(c, data=d) for c, d in zip(R["columns"], cols)]), where="device")
    out = {}
    for name in ("first", "second"):
        if name == "second":
            eng.clear_batch()
        eng.add_queries(qs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = eng.plan(precision=args.precision)
        eng.run()
        eng.fetch_all()
        out[name] = {"ms": (time.perf_counter() - t0) * 1e3, "reorg_ms": info["reorg_ms"],
                     "reorg_reused": bool(info["reorg_reused"]), "plan_ms": info["plan_ms"]}
    eng.close()
    del dev
    return out


def cpu_baseline(args, sample_rows=300_000):
    """The oracle as it stands, on a bounded sample of the same workload (a seeded fact
    relation of ``sample_rows`` tuples with the same dimension relations), timed on the host."""
    from oracle import lmfao_oracle as O
    rels, qs = workload(sample_rows, seed=args.seed, which=args.workload)
    t0 = time.perf_counter()
    O.evaluate(rels, qs)
    dt = time.perf_counter() - t0
    cores = 1  # numpy evaluation of the oracle runs on one host thread
    return {"value": sample_rows / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the whole batch over a seeded {sample_rows}-tuple fact relation of the same shape "
                      f"with the same dimension relations, {dt:.1f} s",
            "host_cpus": os.cpu_count()}


def _family(q, agg):
    """Aggregate family for the error report: grouped or not (and how), and the degree of
    the product (COUNT = 0, SUM(x) = 1, SUM(x_i x_j) = 2, ...)."""
    deg = sum(int(p) if fn == "pow" else 1 for _a, fn, p in agg)
    gb = q.get("groupby", [])
    kind = "ungrouped" if not gb else ("bucketed" if any(k == "bucket" for _a, k, _t in gb) else
                                       f"grouped{len(gb)}")
    if q.get("filters"):
        kind += "+filter"
    return f"{kind}:deg{deg}"


def parity_report(qs, got, ref, oracle_s, processes, chunks):
    """Every aggregate of the engine's results against the chunked FP64/INT64 oracle: group
    keys and counts bit-exact, integral aggregates exact, and per family the largest error
    relative to the sum of absolute terms of the aggregate (the tolerance measure)."""
    fam = {}
    keys_ok = counts_ok = True
    worst = 0.0
    for q, g, r in zip(qs, got, ref):
        if g["keys"].shape != r["keys"].shape or not np.array_equal(g["keys"], r["keys"]):
            keys_ok = False
            continue
        counts_ok &= bool(np.array_equal(g["counts"], r["counts"]))
        for j, agg in enumerate(q["aggs"]):
            name = _family(q, agg)
            f = fam.setdefault(name, {"aggregates": 0, "max_rel_err": 0.0, "exact": True})
            f["aggregates"] += 1
            gj, rj, aj = g["sums"][:, j], r["sums"][:, j], r["abs"][:, j]
            if not agg or all(fn == "ind" for _a, fn, _p in agg):
                f["exact"] &= bool(np.array_equal(gj, rj))
                counts_ok &= bool(np.array_equal(gj, rj))
                continue
            err = np.abs(gj - rj)
            nz = aj > 0
            e = float((err[nz] / aj[nz]).max()) if nz.any() else 0.0
            if (~nz).any() and float(err[~nz].max()) > 1e-9:
                e = float("inf")
            f["max_rel_err"] = max(f["max_rel_err"], e)
            worst = max(worst, e)
    return {"families": fam, "group_keys_equal": keys_ok, "counts_exact": counts_ok, "max_rel_err": worst,
            "tolerance": 1e-5, "within_tolerance": keys_ok and counts_ok and worst <= 1e-5,
            "oracle": "chunked FP64/INT64 oracle over the whole workload", "oracle_chunks": chunks,
            "oracle_cores": processes, "oracle_s": round(oracle_s, 1)}


def full_parity(rels, qs, got):
    from oracle import lmfao_oracle as O
    procs = max(1, os.cpu_count() or 1)
    ref, secs = O.evaluate_chunked(rels, qs, root=0, processes=procs)
    chunks = -(-rels[0]["nrows"] // O.CHUNK)
    return parity_report(qs, got, ref, secs, procs, chunks)


def bench_reference(args):
    """Reference arm: the CPU oracle on a bounded sample per step (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import lmfao_oracle as O
    sample = args.ref_rows
    rels, qs = workload(sample, seed=args.seed, which=args.workload)
    for _ in range(args.warmup):
        O.evaluate(rels, qs)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.evaluate(rels, qs)
        t.append(time.perf_counter() - t0)
    s = float(np.mean(t))
    v = sample / s
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": f"synthetic (seeded, {args.workload}-shaped)",
        "config": workload_config(args, sample, qs),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: the whole batch over a seeded {sample}-tuple fact relation "
                                   f"of the same shape with the same dimension relations"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lmfao", choices=["lmfao", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "split_bf16"])
    ap.add_argument("--workload", default="retailer", choices=sorted(WORKLOADS))
    ap.add_argument("--fact-rows", type=int, default=None)
    ap.add_argument("--ref-rows", type=int, default=200_000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="plan with the default tiles instead of timing candidates")
    ap.add_argument("--no-parity", dest="parity", action="store_false",
                    help="skip the comparison of every aggregate with the oracle over the whole workload")
    args = ap.parse_args()
    if args.fact_rows is None:
        args.fact_rows = WORKLOADS[args.workload][1]
    if args.warmup < 3 and args.impl == "lmfao":
        args.warmup = 3
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_lmfao(args)


if __name__ == "__main__":
    main()
