"""Data-parallel evaluation of one aggregate batch over row shards of a relation.

The rows of one relation (the fact relation, normally the largest) are split into
contiguous, disjoint ranges, one per rank. Every rank holds the other relations whole,
evaluates the same batch over its shard with its own engine on its own GPU, and the ranks
then sum their result states (``Engine.result_state``: int64 counts and integral sums,
float64 sums, in a layout fixed by the batch and the attribute domains) with one
all-reduce. The natural join distributes over a partition of any one of its relations
(the join of the whole is the disjoint union of the joins of the shards), and every
result of a batch is a sum over the join's tuples (Section 2), so the summed state is the
state of the whole relation and ``fetch`` reads it unchanged.

Collectives go through ``torch.distributed`` (NCCL between GPUs; the same code runs on
gloo with CPU tensors). The merge is the only exchange of the path; the dimension views
are computed on every rank from the replicated relations.
"""
from __future__ import annotations


def shard_range(n, rank, world):
    """Rows [lo, hi) of shard ``rank`` of ``world`` balanced contiguous shards of ``n`` rows."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad shard {rank} of {world}")
    return n * rank // world, n * (rank + 1) // world


def shard_relation(rel, rank, world):
    """The relation restricted to its shard's rows (column arrays are views, not copies)."""
    lo, hi = shard_range(int(rel["nrows"]), rank, world)
    cols = [dict(c, data=c["data"][lo:hi]) for c in rel["columns"]]
    return {"name": rel["name"], "nrows": hi - lo, "columns": cols}


def merge_state(counts, sums, group=None):
    """Sum the result state over the ranks of ``group``, in place (two all-reduces: int64 and
    float64). Unsigned 64-bit integral sums wrap the same way as int64 ones, so the int64
    sum is exact modulo 2^64 like the engine's own accumulation."""
    import torch.distributed as dist
    if counts.numel():
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    if sums.numel():
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return counts, sums


class ShardedBatch:
    """One rank's part of a data-parallel batch: its shard of ``shard`` plus every other
    relation, the batch, a plan, and ``run`` = the local evaluation + the merge.

    ``engine_factory(device)`` makes the engine (default: ``lmfao.Engine``); anything with
    ``load_relation``, ``add_queries``, ``plan``, ``run``, ``result_state``, ``fetch_all`` and
    ``close`` serves."""

    def __init__(self, rels, queries, shard=None, rank=None, world=None, group=None, device=0,
                 engine_factory=None):
        import torch.distributed as dist
        if rank is None:
            rank = dist.get_rank(group) if dist.is_initialized() else 0
        if world is None:
            world = dist.get_world_size(group) if dist.is_initialized() else 1
        if shard is None:
            shard = max(rels, key=lambda r: int(r["nrows"]))["name"]
        if shard not in [r["name"] for r in rels]:
            raise ValueError(f"no relation named {shard!r}")
        self.rank, self.world, self.group, self.shard = rank, world, group, shard
        if engine_factory is None:
            from .lmfao import Engine as engine_factory
        self.engine = engine_factory(device)
        try:
            for R in rels:
                self.engine.load_relation(shard_relation(R, rank, world) if R["name"] == shard else R)
            self.engine.add_queries(queries)
        except Exception:
            self.engine.close()
            raise
        self.local_rows = shard_range(int(next(r for r in rels if r["name"] == shard)["nrows"]), rank, world)

    def plan(self, **opts):
        """Plan the local evaluation. The heuristic planner roots the plan at the largest
        relation, which for a shard may no longer be the sharded one: it is rooted at the
        sharded relation instead, as it would be for the whole relation."""
        if opts.get("planner", "heuristic") == "heuristic" and opts.get("root") is None:
            opts["root"] = self.shard
        return self.engine.plan(**opts)

    def run(self, stream=None):
        """Evaluate the local shard on ``stream`` and merge the states of all ranks; the
        all-reduce is ordered after the local run on the same stream."""
        self.engine.run(stream)
        if self.world == 1:
            return
        counts, sums = self.engine.result_state()
        if counts.is_cuda and stream is not None:
            import torch
            with torch.cuda.stream(stream):
                merge_state(counts, sums, self.group)
        else:
            merge_state(counts, sums, self.group)

    def fetch_all(self):
        return self.engine.fetch_all()

    def close(self):
        self.engine.close()
