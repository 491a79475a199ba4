"""The oracle's regression-tree growth (Section 3, decision trees) pinned by brute force: on a
star join whose dimension keys are unique and always present, every fact row is one joined
tuple, so each node's rows can be formed by direct indexing and every candidate split scored
from the node's y values themselves (numpy.var times the count), independently of the
oracle's join, aggregates and bucket arithmetic."""
import numpy as np

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W


def joined_columns(rels):
    F, D1, D2 = rels
    f = {c["attr"]: c["data"] for c in F["columns"]}
    d1 = {c["attr"]: c["data"] for c in D1["columns"]}
    d2 = {c["attr"]: c["data"] for c in D2["columns"]}
    cols = {a: v for a, v in f.items()}
    cols.update({a: v[f["a"]] for a, v in d1.items() if a != "a"})
    cols.update({a: v[f["b"]] for a, v in d2.items() if a != "b"})
    return cols


def brute_tree(cols, target, features, thresholds, depth):
    y = cols[target].astype(np.float64)
    nn = (1 << depth) - 1
    rows = [None] * nn
    rows[0] = np.arange(len(y))
    out = [None] * nn
    for v in range(nn):
        if rows[v] is None:
            continue
        idx = rows[v]
        best = None
        for fi, f in enumerate(features):
            x = cols[f][idx]
            for t in thresholds[f]:
                left = x <= np.float32(t)
                nl, nr = int(left.sum()), int((~left).sum())
                if nl == 0 or nr == 0:
                    continue
                sc = np.var(y[idx][left]) * nl + np.var(y[idx][~left]) * nr
                if best is None or sc < best[2] - 1e-9 * abs(best[2]):
                    best = (fi, float(np.float32(t)), sc)
        out[v] = (len(idx), best)
        if best is not None and 2 * v + 2 < nn:
            x = cols[features[best[0]]][idx]
            rows[2 * v + 1] = idx[x <= np.float32(best[1])]
            rows[2 * v + 2] = idx[x > np.float32(best[1])]
    return out


def test_oracle_tree_equals_brute_force_split_search():
    rels = W.star_schema(n_fact=4000, seed=5)
    feats = ["f1", "f2", "x1", "x2", "x3", "z1", "z2"]
    thr = W.bucket_thresholds(rels, feats, seed=5)
    thr = {f: thr[f][::3] for f in feats}  # 7 thresholds per feature keep the brute force small
    depth = 3
    nodes = O.cart_tree(rels, "y", feats, thr, depth)
    ref = brute_tree(joined_columns(rels), "y", feats, thr, depth)
    for v, (nd, rf) in enumerate(zip(nodes, ref)):
        if rf is None:
            assert not nd["active"], v
            continue
        cnt, best = rf
        assert nd["active"] and nd["count"] == cnt, v
        assert best is not None and nd["feature"] == best[0] and nd["threshold"] == best[1], (v, nd, best)
        assert abs(nd["score"] - best[2]) <= 1e-9 * abs(best[2]), v


def test_best_split_ties_go_to_the_lower_feature_then_threshold():
    """Two identical features give identical scores: the first one wins; within a feature the
    lower threshold wins when two thresholds split the rows identically."""
    keys = np.array([[0], [1], [2], [3]])
    r = {"keys": keys, "counts": np.array([2, 2, 2, 2]),
         "sums": np.array([[0, 2.0, 2.0], [0, 2.0, 2.0], [0, 10.0, 50.0], [0, 10.0, 50.0]])}
    empty_mid = {"keys": np.array([[0], [2], [3]]), "counts": np.array([4, 2, 2]),
                 "sums": np.array([[0, 4.0, 4.0], [0, 10.0, 50.0], [0, 10.0, 50.0]])}
    f, k, sc = O.best_split([r, r], [4, 4])
    assert (f, k) == (0, 1) and abs(sc - 0.0) < 1e-12
    f, k, _ = O.best_split([empty_mid], [4])
    assert (f, k) == (0, 0)  # buckets 0 and 1 split the rows identically; the lower threshold wins
