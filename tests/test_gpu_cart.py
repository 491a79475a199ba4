"""The full CART loop on the GPU (lmfao_cart_tree) against the oracle's tree, and the reuse of
the reorganised root relation across plans over the same relations."""
import numpy as np
import pytest

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W
from paper_2008_08657_b300.lmfao import Engine
from tests.parity import compare

pytestmark = pytest.mark.gpu

FEATS = [a for a in W.RETAILER_CONTS if a != "y"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_depth4_tree_equals_the_oracle_tree(precision):
    """A depth-4 regression tree (15 split decisions, the last level's 8 nodes in one filter
    family) on the Retailer shape with 1M fact tuples: same splits, node counts exact, node
    sums and scores within tolerance of the oracle's."""
    rels = W.retailer_schema(n_fact=1_000_000, seed=3)
    thr = W.bucket_thresholds(rels, FEATS, seed=3)
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    nodes, level_ms = e.cart_tree("y", FEATS, thr, 4, precision=precision)
    e.close()
    ref = O.cart_tree(rels, "y", FEATS, thr, 4, processes=4)
    assert len(level_ms) == 4 and all(p >= 0 and r > 0 for p, r in level_ms)
    for v, (g, r) in enumerate(zip(nodes, ref)):
        assert g["active"] == r["active"], v
        if not r["active"]:
            continue
        assert g["count"] == r["count"], v
        scale = abs(r["sum_y2"]) + 1.0
        assert abs(g["sum_y"] - r["sum_y"]) <= 1e-5 * scale and abs(g["sum_y2"] - r["sum_y2"]) <= 1e-5 * scale, v
        assert (g["feature"], g["threshold"]) == (r["feature"], r["threshold"]), (v, g, r)
        assert abs(g["score"] - r["score"]) <= 1e-5 * scale, (v, g["score"], r["score"])


def test_reorganised_root_is_reused_by_a_new_batch():
    """The second plan over the same relations (a new batch) reuses the segment order of the
    first; results stay oracle-equal."""
    rels = W.retailer_schema(n_fact=300_000, seed=6)
    qs = W.retailer_batch()
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_queries(qs[:2])
    first = e.plan()
    e.run()
    got1 = e.fetch_all()
    e.clear_batch()
    e.add_queries(qs[2:6])
    second = e.plan()
    e.run()
    got2 = e.fetch_all()
    desc = e.describe()["physical"]
    e.close()
    assert first["reorg_reused"] == 0 and first["reorg_ms"] > 0
    assert second["reorg_reused"] == 1 and desc["reorganisation_reused"]
    assert second["reorg_ms"] < first["reorg_ms"]
    ref = O.evaluate(rels, qs[:6])
    for i, (q, g, r) in enumerate(zip(qs[:6], got1 + got2, ref)):
        compare(q, g, r, where=f"query {i}")
