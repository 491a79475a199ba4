"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The Retailer-shaped batch over 84M fact tuples, the Favorita-shaped batch over 120M and the
decision-tree level over 84M run through the C ABI exactly as the benchmark plans them
(FP32, heuristic plan, generated root pass). A seeded sample of their aggregates (every
query keeps its group-by and filters; COUNT and a few sums per query) is evaluated by the
FP64/INT64 oracle over the whole join, in 1M-tuple chunks spread over the host cores, and
compared element by element: group keys and counts bit-exact, sums within 1e-5 of the sum
of absolute terms. At these sizes a segment of the root holds ~520 tuples, so per-segment
FP32 sums, per-CTA partials and the u32 histograms run at the lengths the benchmark sees.
"""
import os

import numpy as np
import pytest

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W
from paper_2008_08657_b300.lmfao import Engine
from tests.parity import compare

pytestmark = pytest.mark.gpu


def sample_batch(qs, seed, per_query=3, max_queries=24):
    """(query index, aggregate indices) pairs: COUNT plus per_query random aggregates of each of
    at most max_queries random queries (the ungrouped query always, with 12 aggregates)."""
    r = np.random.default_rng(seed)
    qidx = list(range(len(qs)))
    if len(qidx) > max_queries:
        qidx = sorted([0] + list(r.choice(np.arange(1, len(qs)), max_queries - 1, replace=False)))
    out = []
    for qi in qidx:
        n = len(qs[qi]["aggs"])
        k = min(n, 12 if qi == 0 else per_query)
        aj = sorted(set([0] + list(r.choice(n, k, replace=False))))
        out.append((qi, aj))
    return out


def run_full(which, n_fact):
    if which == "favorita":
        rels, qs = W.favorita_schema(n_fact=n_fact), W.favorita_batch()
    else:
        rels = W.retailer_schema(n_fact=n_fact)
        qs = W.retailer_batch() if which == "retailer" else W.dt_level_batch(rels)[0]
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_queries(qs)
    e.plan(precision="fp32")
    phys = e.describe()["physical"]
    e.run()
    got = e.fetch_all()
    e.close()
    return rels, qs, got, phys


@pytest.mark.parametrize("which,n_fact", [("retailer", 84_000_000), ("favorita", 120_000_000),
                                          ("dt", 84_000_000)])
def test_full_size_sampled_aggregates_match_the_oracle(which, n_fact):
    rels, qs, got, phys = run_full(which, n_fact)
    assert phys["root_pass"]["generated"], phys["root_pass"]["not_generated_because"]
    picks = sample_batch(qs, seed={"retailer": 1, "favorita": 2, "dt": 3}[which])
    sub = [dict(qs[qi], aggs=[qs[qi]["aggs"][j] for j in aj]) for qi, aj in picks]
    ref, secs = O.evaluate_chunked(rels, sub, root=0, processes=max(1, os.cpu_count() or 1))
    for (qi, aj), q, r in zip(picks, sub, ref):
        g = got[qi]
        g = {"keys": g["keys"], "counts": g["counts"], "sums": g["sums"][:, aj]}
        compare(q, g, r, where=f"{which} query {qi} aggregates {aj}")
