"""Rank bodies of the multi-process tests of the data-parallel merge (gloo, CPU).

``OracleEngine`` stands in for the GPU engine on a CPU rank: it evaluates its shard with the
oracle and keeps the results in a dense state of fixed layout (per query: COUNT per group
cell, then FP64 sums per cell), which is what ``ShardedBatch`` merges. The layout depends
only on the batch and the attribute domains, as the engine's does.
"""
import os
import pickle
from datetime import timedelta

import numpy as np


def _domains(rels, q):
    dom = {}
    for R in rels:
        for c in R["columns"]:
            dom[c["attr"]] = int(c["domain"])
    out = []
    for attr, kind, thr in q.get("groupby", []):
        out.append(len(thr) + 1 if kind == "bucket" else dom[attr])
    return out


class OracleEngine:
    def __init__(self, device=None):
        self.rels, self.queries = [], []

    def load_relation(self, rel, where="host"):
        self.rels.append(rel)

    def add_queries(self, qs):
        self.queries += list(qs)

    def plan(self, **opts):
        import torch
        self.doms = [_domains(self.rels, q) for q in self.queries]
        self.cells = [int(np.prod(d)) if d else 1 for d in self.doms]
        self.io = np.cumsum([0] + self.cells)
        self.fo = np.cumsum([0] + [c * len(q["aggs"]) for c, q in zip(self.cells, self.queries)])
        self.counts = torch.zeros(int(self.io[-1]), dtype=torch.int64)
        self.sums = torch.zeros(int(self.fo[-1]), dtype=torch.float64)
        return {}

    def run(self, stream=None):
        from oracle import lmfao_oracle as O
        self.counts.zero_()
        self.sums.zero_()
        res = O.evaluate(self.rels, self.queries)
        for i, (q, r) in enumerate(zip(self.queries, res)):
            na = len(q["aggs"])
            for key, cnt, s in zip(r["keys"], r["counts"], r["sums"]):
                cell = 0
                for k, d in zip(key, self.doms[i]):
                    cell = cell * d + int(k)
                self.counts[int(self.io[i]) + cell] += int(cnt)
                base = int(self.fo[i]) + cell * na
                self.sums[base:base + na] += np.asarray(s, dtype=np.float64)

    def result_state(self):
        return self.counts, self.sums

    def fetch_all(self):
        out = []
        c, s = self.counts.numpy(), self.sums.numpy()
        for i, q in enumerate(self.queries):
            na, d = len(q["aggs"]), self.doms[i]
            cnt = c[self.io[i]:self.io[i + 1]]
            sm = s[self.fo[i]:self.fo[i + 1]].reshape(-1, na) if na else np.zeros((len(cnt), 0))
            cells = np.nonzero(cnt > 0)[0] if d else np.arange(1)
            keys = np.zeros((len(cells), len(d)), dtype=np.int64)
            rem = cells.copy()
            for j in range(len(d) - 1, -1, -1):
                keys[:, j] = rem % d[j]
                rem //= d[j]
            out.append({"keys": keys, "counts": cnt[cells].astype(np.int64), "sums": sm[cells]})
        return out

    def close(self):
        pass


def _init(rank, world, port, timeout_s=60):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=timeout_s))


def merge_rank(rank, world, port, workload_path, out_dir):
    """Each rank evaluates its shard of F and merges; every rank writes its fetched results."""
    import torch.distributed as dist
    from paper_2008_08657_b300.distributed import ShardedBatch
    _init(rank, world, port)
    with open(workload_path, "rb") as f:
        rels, qs = pickle.load(f)
    b = ShardedBatch(rels, qs, shard="F", engine_factory=OracleEngine)
    b.plan()
    b.run()
    res = b.fetch_all()
    with open(os.path.join(out_dir, f"rank{rank}.pkl"), "wb") as f:
        pickle.dump({"results": res, "rows": b.local_rows}, f)
    dist.barrier()
    dist.destroy_process_group()


def failing_rank(rank, world, port, workload_path, out_dir):
    """Rank 1 fails between steps (before the merge); rank 0 must get an error from its
    merge, not wait forever."""
    import torch.distributed as dist
    from paper_2008_08657_b300.distributed import ShardedBatch
    _init(rank, world, port, timeout_s=5)
    with open(workload_path, "rb") as f:
        rels, qs = pickle.load(f)
    b = ShardedBatch(rels, qs, shard="F", engine_factory=OracleEngine)
    b.plan()
    if rank == 1:
        raise SystemExit(3)
    status = "merged"
    try:
        b.run()
    except Exception as e:  # the peer is gone: the collective reports it
        status = "error: " + type(e).__name__
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(status)
    try:
        dist.destroy_process_group()
    except Exception:
        pass
