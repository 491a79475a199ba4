"""COUNT GROUP BY with hash-table results (lmfao_group_count; Rk-means steps 1 and 3 of
Section 3) against the oracle: groups and counts bit-exact, for value, bucket and FP32-value
group attributes homed at the root and at dimension relations."""
import numpy as np
import pytest

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W
from paper_2008_08657_b300.lmfao import ERR_UNSUPPORTED, Engine, LmfaoError

pytestmark = pytest.mark.gpu


def _grid(rels, attrs, k, seed):
    """Cluster intervals of a stand-in for Rk-means step 2: k seeded quantile centroids per
    attribute; the grid cell of a value is the number of midpoints strictly below it."""
    r = np.random.default_rng(seed)
    out = []
    for a in attrs:
        v = next(c["data"] for R in rels for c in R["columns"] if c["attr"] == a).astype(np.float64)
        cents = np.sort(np.quantile(v, np.sort(r.uniform(0.05, 0.95, k))))
        mids = np.unique(((cents[1:] + cents[:-1]) / 2).astype(np.float32))
        out.append((a, "bucket", mids))
    return out


def _check(rels, gb, cap=None):
    q = {"aggs": [[]], "groupby": gb, "filters": []}
    ref = O.evaluate(rels, [q])[0]
    e = Engine(0)
    try:
        for R in rels:
            e.load_relation(R)
        keys, counts, n = e.group_count([(a, "value" if kind == "float" else kind, t) for a, kind, t in gb],
                                        cap or len(ref["keys"]) + 10)
    finally:
        e.close()
    assert n == len(ref["keys"])
    order = np.lexsort(keys.T[::-1])
    np.testing.assert_array_equal(keys[order], ref["keys"])
    np.testing.assert_array_equal(counts[order], ref["counts"])


@pytest.mark.parametrize("attr", ["x1", "z2", "f1", "c1"])
def test_rk_means_step1_counts_per_value(attr):
    """SUM(1) GROUP BY X_j: the values of a dimension feature, of a fact feature (one group per
    distinct FP32 value) and of a categorical."""
    rels = W.star_schema(n_fact=200_000, seed=3)
    kind = "value" if attr == "c1" else "float"
    _check(rels, [(attr, kind, None)])


@pytest.mark.parametrize("which", ["star", "retailer"])
def test_rk_means_step3_grid_coreset(which):
    """SUM(1) GROUP BY C_1..C_n over a grid of cluster intervals of attributes of every relation."""
    if which == "star":
        rels = W.star_schema(n_fact=200_000, seed=4)
        attrs = ["y", "f1", "x1", "x2", "z1", "z2"]
    else:
        rels = W.retailer_schema(n_fact=1_000_000, seed=4)
        attrs = ["y", "i1", "i2", "l1", "c3", "w1", "w5"]
    _check(rels, _grid(rels, attrs, 6, seed=5))


def test_group_count_reports_the_true_number_past_the_capacity_and_refuses_wide_keys():
    rels = W.star_schema(n_fact=50_000, seed=6)
    e = Engine(0)
    try:
        for R in rels:
            e.load_relation(R)
        keys, counts, n = e.group_count([("f1", "value", None)], 100)
        f1 = rels[0]["columns"][3]["data"]
        assert n == len(np.unique(f1.view(np.uint32))) and len(keys) == 100 and counts.sum() >= 100
        with pytest.raises(LmfaoError) as ei:
            e.group_count([("f1", "value", None), ("f2", "value", None)], 10)
        assert ei.value.code == ERR_UNSUPPORTED
    finally:
        e.close()
