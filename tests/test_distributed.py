"""Data-parallel merge over row shards (multi-process, gloo on CPU).

Ranks evaluate disjoint contiguous shards of the fact relation and sum their result states;
the merged results equal the oracle's over the whole relation (the join distributes over a
partition of one of its relations, and every result is a sum over the join). A rank that
fails between steps makes the others' merge raise instead of waiting.
"""
import os
import pickle
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W
from paper_2008_08657_b300.distributed import shard_range, shard_relation
from tests import dist_worker
from tests.parity import compare


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (7, 3), (1000, 4), (10, 16)])
def test_shards_cover_the_rows_once_in_order(n, world):
    ranges = [shard_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a <= b
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_shard_relation_slices_every_column():
    F = W.star_schema(n_fact=101, seed=3)[0]
    parts = [shard_relation(F, r, 3) for r in range(3)]
    assert sum(p["nrows"] for p in parts) == 101
    for j, c in enumerate(F["columns"]):
        np.testing.assert_array_equal(np.concatenate([p["columns"][j]["data"] for p in parts]), c["data"])


def _spawn(fn, world, rels, qs, tmp_path):
    path = os.path.join(tmp_path, "workload.pkl")
    with open(path, "wb") as f:
        pickle.dump((rels, qs), f)
    ctx = mp.get_context("spawn")
    port = _port()
    procs = [ctx.Process(target=fn, args=(r, world, port, path, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    return [p.exitcode for p in procs]


def _star():
    rels = W.star_schema(n_fact=3000, seed=5, n_d1=40, n_d2=30)
    return rels, W.star_batch()


def _dangling():
    # tiny schema with dangling and repeated keys; the fact relation renamed F for sharding
    rels = W.tiny_schema(11, max_rows=40, kdom=6, shared3=True, fd=True)
    rels = [dict(R, name="F") if R["name"] == "R0" else R for R in rels]
    qs = W.tiny_queries(11, rels, nq=5, group_attrs=["k1", "k2", "g0", "g1"], bucket_attrs=["x0", "x1"])
    return rels, qs


@pytest.mark.parametrize("make,world", [(_star, 2), (_dangling, 2), (_dangling, 3)])
def test_merged_shards_equal_the_whole_relation(make, world, tmp_path):
    rels, qs = make()
    codes = _spawn(dist_worker.merge_rank, world, rels, qs, tmp_path)
    assert codes == [0] * world
    ref = O.evaluate(rels, qs)
    n = next(R for R in rels if R["name"] == "F")["nrows"]
    for r in range(world):
        with open(os.path.join(tmp_path, f"rank{r}.pkl"), "rb") as f:
            got = pickle.load(f)
        assert tuple(got["rows"]) == shard_range(n, r, world)
        for i, (q, g, e) in enumerate(zip(qs, got["results"], ref)):
            compare(q, g, e, where=f"rank {r} query {i}")


def test_a_failed_rank_makes_the_merge_raise(tmp_path):
    rels, qs = _star()
    codes = _spawn(dist_worker.failing_rank, 2, rels, qs, tmp_path)
    assert codes[1] == 3
    with open(os.path.join(tmp_path, "rank0.txt")) as f:
        assert f.read().startswith("error")
