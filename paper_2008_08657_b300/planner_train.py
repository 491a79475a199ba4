"""Learned planner: measured plan times -> MLP cost model -> regret.

For each seeded random snowflake schema (3-8 relations, uniform or Zipf(1.1) keys, 2-12
float features per relation) with a ridge + group-by batch of the star-join kind (8
continuous attributes spread over the relations and up to 2 categoricals):

1. ``lmfao_plan_candidates`` lists the candidate physical plans (root relation, segment
   relation, root pass, combine) with their features;
2. every candidate is planned (FORCED) and timed with CUDA events (median of a few runs);
   the best measured time is the exhaustive planner's choice;
3. the cost model (3 x 64 MLP, ``CostModel``: forward, backward and Adam run in the
   engine's CUDA kernels) is trained on log-times of the training schemas;
4. on held-out schemas the learned choice (argmin of the predicted time) and the
   heuristic choice (default plan) are compared with the exhaustive one:
   regret = t(choice) / t(best) - 1.

Usage: ``python -m paper_2008_08657_b300.planner_train --schemas 300 --train 200 --out DIR``
writes DIR/planner_data.npz, DIR/cost_model.txt and DIR/planner_results.json.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import workloads as W
from .lmfao import COST_MODEL_PATH, CostModel, Engine, LmfaoError


def schema_batch(seed, fact_range=(1e5, 5e6), n_conts=8, n_cats=2):
    """A random snowflake and its ridge + group-by batch (seeded)."""
    rels, parents, conts, cats = W.random_snowflake(seed, fact_range=fact_range)
    r = np.random.default_rng(np.random.SeedSequence([seed, 77]))
    pick = sorted(r.choice(len(conts), min(n_conts, len(conts)), replace=False))
    cpick = sorted(r.choice(len(cats), min(n_cats, len(cats)), replace=False)) if cats else []
    qs = W.ridge_batch([conts[i] for i in pick], [cats[i] for i in cpick])
    return rels, qs


def time_current_plan(eng, torch, stream, reps=5, warm=2):
    for _ in range(warm):
        eng.run(stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    for i in range(reps):
        ev[2 * i].record(stream)
        eng.run(stream)
        ev[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    return float(np.median([ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps)]))


def measure_schema(seed, torch, stream, fact_range=(1e5, 5e6), reps=5):
    """Features and measured times of every candidate plan, and the heuristic plan's time."""
    rels, qs = schema_batch(seed, fact_range)
    eng = Engine(0)
    try:
        for R in rels:
            eng.load_relation(R)
        eng.add_queries(qs)
        cands, feats = eng.plan_candidates()
        times = np.full(len(cands), np.inf)
        for i, c in enumerate(cands):
            try:
                eng.plan_candidate(c)
                t = time_current_plan(eng, torch, stream, reps)
                eng.fetch(0)  # raises when the plan's device checks fail on this data
                times[i] = t
            except LmfaoError:
                pass
        try:
            eng.plan()
            t_heur = time_current_plan(eng, torch, stream, reps)
            eng.fetch(0)
        except LmfaoError:
            t_heur = np.inf
    finally:
        eng.close()
    return {"seed": seed, "cands": cands, "feats": feats, "times": times, "t_heur": t_heur,
            "fact_rows": rels[0]["nrows"], "relations": len(rels)}


def collect(seeds, fact_range=(1e5, 5e6), log=None):
    import torch
    stream = torch.cuda.Stream()
    out = []
    for k, s in enumerate(seeds):
        out.append(measure_schema(s, torch, stream, fact_range))
        if log and (k + 1) % 20 == 0:
            log(f"measured {k + 1}/{len(seeds)} schemas")
    return out


def stack(data):
    X, y, g = [], [], []
    for i, d in enumerate(data):
        ok = np.isfinite(d["times"])
        X.append(d["feats"][ok])
        y.append(np.log(d["times"][ok]))
        g.append(np.full(ok.sum(), i))
    return np.concatenate(X), np.concatenate(y), np.concatenate(g)


def _normaliser(data):
    X, _, _ = stack(data)
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std[std < 1e-6] = 1.0
    return mean, std


def _fit(data, mean, std, steps, lr, seed, check=None, every=250):
    """Train one model; with ``check`` (a callable on the model), record it every ``every`` steps."""
    import torch
    X, y, _ = stack(data)
    model = CostModel(X.shape[1], seed=seed)
    xt = torch.tensor((X - mean) / std, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    trace = []
    for k in range(1, steps + 1):
        model.train_step(xt, yt, lr=lr)
        if check is not None and k % every == 0:
            trace.append((k, check(model)))
    return model, trace


def train(data, max_steps=3000, lr=2e-3, members=5, val_frac=0.2, seed=0):
    """Choose the number of training steps on a validation split of the training schemas
    (mean regret of the learned choice), then train an ensemble of ``members`` models on all
    training schemas; the prediction is the ensemble mean."""
    nval = max(1, int(len(data) * val_frac))
    fit_part, val_part = data[:-nval], data[-nval:]
    mean, std = _normaliser(fit_part)
    _, trace = _fit(fit_part, mean, std, max_steps, lr, seed, check=lambda m: regrets(val_part, [m], mean, std)[0].mean())
    best_steps = min(trace, key=lambda kv: kv[1])[0]
    mean, std = _normaliser(data)
    models = [_fit(data, mean, std, best_steps, lr, seed + 1 + i)[0] for i in range(members)]
    return models, mean, std, {"validation_trace": trace, "steps": best_steps}


def save_model(path, models, mean, std):
    with open(path, "w") as f:
        f.write(f"lmfao-cost-model 2 {models[0].d} {len(models)}\n")
        f.write(" ".join(f"{v:.9g}" for v in mean) + "\n")
        f.write(" ".join(f"{v:.9g}" for v in std) + "\n")
        for m in models:
            f.write(" ".join(f"{v:.9g}" for v in m.params.cpu().numpy()) + "\n")


def load_model(path):
    import torch
    with open(path) as f:
        head = f.readline().split()
        d, k = int(head[2]), int(head[3])
        mean = np.array(f.readline().split(), dtype=np.float64)
        std = np.array(f.readline().split(), dtype=np.float64)
        models = []
        for _ in range(k):
            p = np.array(f.readline().split(), dtype=np.float32)
            m = CostModel(d)
            m.params.copy_(torch.tensor(p))
            models.append(m)
    return models, mean, std


def predict(models, feats, mean, std):
    import torch
    x = torch.tensor((feats - mean) / std, dtype=torch.float32, device="cuda")
    return np.mean([m.forward(x).cpu().numpy() for m in models], axis=0)


def regrets(data, models, mean, std):
    """Per schema: regret of the learned choice and of the heuristic plan."""
    rl, rh = [], []
    for d in data:
        t = d["times"]
        ok = np.isfinite(t)
        if not ok.any():
            continue
        best = t[ok].min()
        pred = predict(models, d["feats"], mean, std)
        pred[~ok] = np.inf
        choice = int(np.argmin(pred))
        rl.append(t[choice] / best - 1.0)
        rh.append(d["t_heur"] / best - 1.0)  # inf when the heuristic plan fails its checks
    return np.array(rl), np.array(rh)


def topk_regrets(data, models, mean, std, k):
    """Per schema: regret of timing the k best-predicted candidates (that pass their checks)
    and keeping the fastest, the LEARNED planner with learned_topk = k."""
    r = []
    for d in data:
        t = d["times"]
        ok = np.isfinite(t)
        if not ok.any():
            continue
        pred = predict(models, d["feats"], mean, std)
        pred[~ok] = np.inf
        picks = [int(c) for c in np.argsort(pred, kind="stable")[:k] if ok[c]]
        r.append(min(t[c] for c in picks) / t[ok].min() - 1.0)
    return np.array(r)


def summarise(tr, te, models, mean, std, extra):
    rl, rh = regrets(te, models, mean, std)
    rl_tr, rh_tr = regrets(tr, models, mean, std)
    res = dict(extra)
    res.update({
        "test_regret_learned_mean": float(rl.mean()), "test_regret_learned_median": float(np.median(rl)),
        "test_regret_learned_p90": float(np.quantile(rl, 0.9)),
        "test_regret_heuristic_mean": float(rh[np.isfinite(rh)].mean()),
        "test_regret_heuristic_median": float(np.median(rh)),
        "test_regret_heuristic_p90": float(np.quantile(rh, 0.9)),
        "test_heuristic_plan_failed": float(np.mean(~np.isfinite(rh))),
        "test_within_10pct_learned": float(np.mean(rl <= 0.10)),
        "test_within_10pct_heuristic": float(np.mean(rh <= 0.10)),
        "train_regret_learned_mean": float(rl_tr.mean()),
        "train_regret_heuristic_mean": float(rh_tr[np.isfinite(rh_tr)].mean()),
        "test_regret_learned_topk": {},
    })
    for k in (2, 3, 4, 5):
        rk = topk_regrets(te, models, mean, std, k)
        res["test_regret_learned_topk"][str(k)] = {
            "mean": float(rk.mean()), "median": float(np.median(rk)), "p90": float(np.quantile(rk, 0.9)),
            "within_10pct": float(np.mean(rk <= 0.10)),
            "candidates_timed_fraction": float(np.mean([min(k, np.isfinite(d["times"]).sum()) / len(d["times"])
                                                        for d in te]))}
    return res


def load_data(path):
    z = np.load(path)
    out = []
    for i, seed in enumerate(z["seeds"]):
        out.append({"seed": int(seed), "cands": z[f"cands_{i}"], "feats": z[f"feats_{i}"], "times": z[f"times_{i}"],
                    "t_heur": float(z["t_heur"][i])})
    return out


def install(out):
    """Copy the trained model and its results into the package (the installed cost model)."""
    import shutil
    here = os.path.dirname(os.path.abspath(__file__))
    shutil.copy(os.path.join(out, "cost_model.txt"), COST_MODEL_PATH)
    shutil.copy(os.path.join(out, "planner_results.json"), os.path.join(here, "planner_results.json"))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--schemas", type=int, default=300)
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--fact-min", type=float, default=1e5)
    ap.add_argument("--fact-max", type=float, default=5e6)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default="planner_out")
    ap.add_argument("--evaluate", action="store_true",
                    help="recompute the results of the data and model already in --out (no measurement)")
    ap.add_argument("--install", action="store_true",
                    help="copy the model and its results into the package as the installed cost model")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    if args.evaluate:
        data = load_data(os.path.join(args.out, "planner_data.npz"))
        models, mean, std = load_model(os.path.join(args.out, "cost_model.txt"))
        with open(os.path.join(args.out, "planner_results.json")) as f:
            old = json.load(f)
        keep = {k: old[k] for k in ("schemas", "train", "test", "fact_rows_range", "candidates_per_schema",
                                    "collect_seconds", "training", "ensemble") if k in old}
        res = summarise(data[:args.train], data[args.train:], models, mean, std, keep)
    else:
        t0 = time.time()
        data = collect(range(args.schemas), (args.fact_min, args.fact_max), log=print)
        t1 = time.time()
        np.savez_compressed(os.path.join(args.out, "planner_data.npz"),
                            **{f"{k}_{i}": v for i, d in enumerate(data) for k, v in d.items()
                               if isinstance(v, np.ndarray)},
                            t_heur=np.array([d["t_heur"] for d in data]),
                            seeds=np.array([d["seed"] for d in data]))
        tr, te = data[:args.train], data[args.train:]
        models, mean, std, info = train(tr, max_steps=args.steps)
        save_model(os.path.join(args.out, "cost_model.txt"), models, mean, std)
        res = summarise(tr, te, models, mean, std, {
            "schemas": args.schemas, "train": len(tr), "test": len(te),
            "fact_rows_range": [args.fact_min, args.fact_max],
            "candidates_per_schema": float(np.mean([len(d["cands"]) for d in data])),
            "collect_seconds": t1 - t0, "training": info, "ensemble": len(models)})
    with open(os.path.join(args.out, "planner_results.json"), "w") as f:
        json.dump(res, f, indent=1)
    if args.install:
        install(args.out)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
