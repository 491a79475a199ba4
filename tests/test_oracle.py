"""Pins of the CPU oracle against things other than itself.

* brute force: nested loops over the cross product of tiny relations (duplicate and
  dangling keys, an attribute shared by three relations), each joined tuple evaluated in
  plain Python floats -- the definition of a group-by aggregate over a natural join
  (Section 1, Section 2);
* invariants: COUNT = |F| for an FK star join with no dangling keys; the groups of a
  group-by sum to the ungrouped aggregate; Sigma is symmetric positive semidefinite
  (Section 3, ridge regression);
* closed forms: the ridge solution from Sigma equals ``numpy.linalg.lstsq`` on the
  materialised design matrix; the CART variance equals ``numpy.var * |T|`` (Section 3);
* an independent method: the factorised view computation of Section 2 (views along the
  join tree of Fig. 2, the loop nest of Fig. 3 with lookups once per key) written out
  here on a small Favorita-shaped instance;
* join-order independence.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W

OPS = {"le": lambda a, b: a <= b, "lt": lambda a, b: a < b, "ge": lambda a, b: a >= b,
       "gt": lambda a, b: a > b, "eq": lambda a, b: a == b, "ne": lambda a, b: a != b}


def brute_force(rels, q):
    """Enumerate the cross product, keep combinations that agree on every shared attribute."""
    ranges = [range(R["nrows"]) for R in rels]
    cols = [{c["attr"]: c for c in R["columns"]} for R in rels]
    out = {}
    for combo in itertools.product(*ranges):
        vals = {}
        ok = True
        for ri, row in enumerate(combo):
            for a, c in cols[ri].items():
                v = c["data"][row]
                if a in vals and vals[a] != v:
                    ok = False
                    break
                vals.setdefault(a, v)
            if not ok:
                break
        if not ok:
            continue
        if not all(OPS[op](float(vals[a]), float(np.float32(t))) for a, op, t in q["filters"]):
            continue
        key = []
        for a, kind, thr in q["groupby"]:
            if kind == "value":
                key.append(int(vals[a]))
            else:
                key.append(sum(1 for t in thr if float(t) < float(vals[a])))
        key = tuple(key)
        terms = []
        for agg in q["aggs"]:
            t = 1.0
            for a, fn, p in agg:
                x = float(vals[a])
                t *= x if fn == "id" else x ** int(p)
            terms.append(t)
        cnt, s = out.get(key, (0, [0.0] * len(terms)))
        out[key] = (cnt + 1, [u + v for u, v in zip(s, terms)])
    if not q["groupby"] and () not in out:
        out[()] = (0, [0.0] * len(q["aggs"]))
    return out


def assert_matches_brute(res, bf, rtol=1e-12):
    keys = [tuple(int(v) for v in k) for k in res["keys"]]
    assert keys == sorted(bf.keys())
    for i, k in enumerate(keys):
        cnt, sums = bf[k]
        assert res["counts"][i] == cnt
        for j, s in enumerate(sums):
            assert abs(res["sums"][i, j] - s) <= rtol * max(1.0, res["abs"][i, j])


@pytest.mark.parametrize("seed", range(40))
def test_oracle_matches_brute_force(seed):
    rels = W.tiny_schema(seed, shared3=(seed % 2 == 1))
    qs = W.tiny_queries(seed, rels, nq=5)
    res = O.evaluate(rels, qs)
    for q, r in zip(qs, res):
        assert_matches_brute(r, brute_force(rels, q))


def test_brute_force_sees_duplicates_and_dangling_keys():
    # the tiny generator must actually exercise many-to-many and unmatched keys
    dup = dangling = 0
    for seed in range(20):
        rels = W.tiny_schema(seed)
        k1 = [rels[0]["columns"][0]["data"], rels[1]["columns"][0]["data"]]
        dup += int(len(set(k1[1].tolist())) < len(k1[1]))
        dangling += int(bool(set(k1[0].tolist()) - set(k1[1].tolist())))
    assert dup > 5 and dangling > 5


def test_count_equals_fact_rows_for_fk_star():
    rels = W.star_schema(n_fact=20_000)
    r = O.evaluate(rels, W.star_batch())
    assert r[0]["counts"][0] == 20_000
    assert r[0]["sums"][0, 0] == 20_000.0


def test_groups_sum_to_ungrouped():
    rels = W.star_schema(n_fact=20_000)
    qs = W.star_batch()
    res = O.evaluate(rels, qs)
    total = res[0]
    conts = W.STAR_CONTS
    for q, r in zip(qs[1:], res[1:]):
        assert r["counts"].sum() == total["counts"][0]
        if len(q["aggs"]) > 1:
            for j, x in enumerate(conts):
                np.testing.assert_allclose(r["sums"][:, 1 + j].sum(), total["sums"][0, 1 + j],
                                           rtol=1e-12, atol=1e-9)


def sigma_from_ridge(res, conts):
    """Assemble Sigma (intercept first) from the ungrouped ridge query (Section 3)."""
    n = len(conts) + 1
    S = np.zeros((n, n))
    s = res["sums"][0]
    S[0, 0] = s[0]
    for i in range(len(conts)):
        S[0, i + 1] = S[i + 1, 0] = s[1 + i]
    k = 1 + len(conts)
    for i in range(len(conts)):
        for j in range(i, len(conts)):
            S[i + 1, j + 1] = S[j + 1, i + 1] = s[k]
            k += 1
    return S


def test_sigma_symmetric_psd():
    rels = W.star_schema(n_fact=20_000)
    res = O.evaluate(rels, W.star_batch())
    S = sigma_from_ridge(res[0], W.STAR_CONTS)
    assert np.allclose(S, S.T)
    np.linalg.cholesky(S + 1e-9 * np.trace(S) * np.eye(len(S)))
    assert np.linalg.eigvalsh(S).min() > -1e-9 * np.trace(S)


def materialise(rels):
    """The join as a list of attribute dicts, by brute force (independent of the oracle)."""
    cols = [{c["attr"]: c for c in R["columns"]} for R in rels]
    rows = []
    for combo in itertools.product(*[range(R["nrows"]) for R in rels]):
        vals = {}
        ok = True
        for ri, row in enumerate(combo):
            for a, c in cols[ri].items():
                v = c["data"][row]
                if a in vals and vals[a] != v:
                    ok = False
                    break
                vals.setdefault(a, v)
            if not ok:
                break
        if ok:
            rows.append(vals)
    return rows


def test_ridge_closed_form_matches_lstsq():
    # y is the label x_n with parameter -1; the model over (1, x0..x3) solves
    # (Sigma_xx + lam I) theta = Sigma_xy (gradient of J in Section 3 set to zero, scaled by |D|)
    rels = W.tiny_schema(3, max_rows=10, empty_ok=False)
    conts = ["x0", "x1", "x2", "x3"]
    label = "x3"
    feats = ["x0", "x1", "x2"]
    q = W.ridge_batch(conts, [])[0]
    S = sigma_from_ridge(O.evaluate(rels, [q])[0], conts)
    idx = [0] + [1 + conts.index(f) for f in feats]
    yi = 1 + conts.index(label)
    lam = 0.5
    A = S[np.ix_(idx, idx)] + lam * np.eye(len(idx))
    theta = np.linalg.solve(A, S[idx, yi])
    rows = materialise(rels)
    assert len(rows) > 3
    X = np.array([[1.0] + [float(r[f]) for f in feats] for r in rows])
    y = np.array([float(r[label]) for r in rows])
    Xa = np.vstack([X, math.sqrt(lam) * np.eye(len(idx))])
    ya = np.concatenate([y, np.zeros(len(idx))])
    ref, *_ = np.linalg.lstsq(Xa, ya, rcond=None)
    np.testing.assert_allclose(theta, ref, rtol=1e-9, atol=1e-9)


def test_cart_variance_matches_numpy_var():
    rels = W.tiny_schema(5, max_rows=12, empty_ok=False)
    thr = np.array([-1.0, 0.0, 0.5], dtype=np.float32)
    q = {"aggs": [[], [("x2", "id", 1)], [("x2", "pow", 2)]],
         "groupby": [("x0", "bucket", thr)], "filters": [("x1", "le", 1.0)]}
    res = O.evaluate(rels, [q])[0]
    rows = [r for r in materialise(rels) if float(r["x1"]) <= 1.0]
    left, right = O.cart_variances(res)
    nb = int(res["keys"][:, 0].max()) + 1
    for k in range(nb - 1):
        tk = float(thr[k])
        L = np.array([float(r["x2"]) for r in rows if float(r["x0"]) <= tk])
        Rr = np.array([float(r["x2"]) for r in rows if float(r["x0"]) > tk])
        assert abs(left[k] - (np.var(L) * len(L) if len(L) else 0.0)) < 1e-9
        assert abs(right[k] - (np.var(Rr) * len(Rr) if len(Rr) else 0.0)) < 1e-9


def test_join_order_does_not_matter():
    rels = W.tiny_schema(11, shared3=True, empty_ok=False)
    qs = W.tiny_queries(11, rels, nq=4)
    a = O.evaluate(rels, qs)
    for order in ([4, 2, 0, 3, 1], [3, 2, 0, 1, 4], [1, 4, 0, 2, 3]):
        b = O.evaluate(rels, qs, order=order)
        for ra, rb in zip(a, b):
            np.testing.assert_array_equal(ra["keys"], rb["keys"])
            np.testing.assert_array_equal(ra["counts"], rb["counts"])
            np.testing.assert_allclose(ra["sums"], rb["sums"], rtol=1e-12, atol=1e-12)


def test_oracle_against_views_of_section_2_favorita():
    """Q1-Q3 of Section 2 computed from directional views along the join tree of Fig. 2
    instead of the materialised join.

    A view from relation X toward its neighbour Y is the aggregate over the part of the join
    on X's side of the edge, grouped by the attributes X shares with Y (Section 2, views);
    here each one is a numpy group-by sum over X's tuples weighted by the views into X.
    Q1 and Q2 (rooted at Sales) weight every Sales tuple by the product of the views into
    Sales; Q3 (rooted at Items) groups by class the view from Sales to Items, which carries
    SUM(units * price) over everything on the Sales side of that edge.
    """
    rels = W.favorita_schema(n_fact=3000, seed=4)
    S, T, R, Oi, H, I = rels
    q = W.favorita_example_queries()
    res = O.evaluate(rels, q)

    def cols(X):
        return {c["attr"]: c["data"] for c in X["columns"]}

    s, t, r, o, h, it = map(cols, (S, T, R, Oi, H, I))
    nd, ns, ni = W.N_FDATE, W.N_STORE, W.N_FITEM
    # views toward Transactions: StoRes by store (COUNT), Oil by date (COUNT, SUM(price))
    r_cnt = np.bincount(r["store"], minlength=ns).astype(float)
    o_cnt = np.bincount(o["date"], minlength=nd).astype(float)
    o_price = np.bincount(o["date"], weights=o["price"].astype(float), minlength=nd)
    # view Transactions -> Sales by (date, store): COUNT and SUM(price) over T, R, O
    tkey = t["date"].astype(np.int64) * ns + t["store"]
    tw = r_cnt[t["store"]]
    t_cnt = np.bincount(tkey, weights=tw * o_cnt[t["date"]], minlength=nd * ns)
    t_price = np.bincount(tkey, weights=tw * o_price[t["date"]], minlength=nd * ns)
    # views Holidays -> Sales by date and Items -> Sales by item (COUNT)
    h_cnt = np.bincount(h["date"], minlength=nd).astype(float)
    i_cnt = np.bincount(it["item"], minlength=ni).astype(float)
    # at Sales: every Sales tuple occurs (product of the COUNT views into Sales) times in D
    skey = s["date"].astype(np.int64) * ns + s["store"]
    units = s["units"].astype(float)
    mult = i_cnt[s["item"]] * h_cnt[s["date"]] * t_cnt[skey]
    Q1 = float((units * mult).sum())
    gdate = s["item"].astype(float) * s["date"].astype(float)
    q2_cnt = np.bincount(s["store"], weights=mult, minlength=ns)
    q2_sum = np.bincount(s["store"], weights=gdate * mult, minlength=ns)
    # view Sales -> Items by item: COUNT and SUM(units * price) over Sales, T, R, O, H
    side = h_cnt[s["date"]]
    si_cnt = np.bincount(s["item"], weights=side * t_cnt[skey], minlength=ni)
    si_up = np.bincount(s["item"], weights=units * side * t_price[skey], minlength=ni)
    # at Items: Q3 GROUP BY class
    q3_cnt = np.bincount(it["class"], weights=si_cnt[it["item"]], minlength=337)
    q3_sum = np.bincount(it["class"], weights=si_up[it["item"]], minlength=337)

    assert abs(res[0]["sums"][0, 0] - Q1) <= 1e-9 * res[0]["abs"][0, 0]
    assert res[0]["counts"][0] == int(round(mult.sum()))
    keys2 = [int(k[0]) for k in res[1]["keys"]]
    assert keys2 == [int(k) for k in np.nonzero(q2_cnt)[0]]
    for g, k in enumerate(keys2):
        assert res[1]["counts"][g] == int(round(q2_cnt[k]))
        assert abs(res[1]["sums"][g, 0] - q2_sum[k]) <= 1e-9 * max(1.0, res[1]["abs"][g, 0])
    keys3 = [int(k[0]) for k in res[2]["keys"]]
    assert keys3 == [int(k) for k in np.nonzero(q3_cnt)[0]]
    for g, k in enumerate(keys3):
        assert res[2]["counts"][g] == int(round(q3_cnt[k]))
        assert abs(res[2]["sums"][g, 0] - q3_sum[k]) <= 1e-9 * max(1.0, res[2]["abs"][g, 0])


def test_planted_mistake_is_caught():
    """A dropped factor in the oracle's product must fail the brute-force pin."""
    rels = W.tiny_schema(2, empty_ok=False)
    q = {"aggs": [[("x0", "id", 1), ("x1", "id", 1)]], "groupby": [], "filters": []}
    good = O.evaluate(rels, [q])[0]
    bad_q = {"aggs": [[("x0", "id", 1)]], "groupby": [], "filters": []}
    bad = O.evaluate(rels, [bad_q])[0]
    bf = brute_force(rels, q)
    assert_matches_brute(good, bf)
    with pytest.raises(AssertionError):
        assert_matches_brute(bad, bf)


@pytest.mark.parametrize("processes", [1, 3])
def test_chunked_evaluation_equals_the_whole_join(processes):
    """The join distributes over a partition of the fact relation: the chunked evaluation
    (chunks summed in order, optionally over spawned processes) gives the same groups and
    counts as the unchunked one, and sums equal up to rounding order; chunks that contribute
    nothing to a group, empty chunks and a ragged last chunk are covered."""
    rels = W.star_schema(n_fact=5003, seed=3)
    qs = W.star_batch() + [{"aggs": [[], [("y", "id", 1)]], "groupby": [("c1", "value", None)],
                            "filters": [("y", "gt", 1.5)]}]
    whole = O.evaluate(rels, qs)
    got, secs = O.evaluate_chunked(rels, qs, root=0, processes=processes, chunk=1000)
    assert secs >= 0
    for a, b in zip(got, whole):
        np.testing.assert_array_equal(a["keys"], b["keys"])
        np.testing.assert_array_equal(a["counts"], b["counts"])
        np.testing.assert_allclose(a["sums"], b["sums"], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(a["abs"], b["abs"], rtol=1e-12, atol=1e-12)
    # the tiny brute-force schemas (duplicate and dangling keys) split into 4-row chunks
    for seed in range(6):
        rels = W.tiny_schema(seed, empty_ok=False)
        qs = W.tiny_queries(seed, rels, nq=3)
        whole = O.evaluate(rels, qs)
        got, _ = O.evaluate_chunked(rels, qs, root=0, processes=1, chunk=4)
        for a, b in zip(got, whole):
            np.testing.assert_array_equal(a["keys"], b["keys"])
            np.testing.assert_array_equal(a["counts"], b["counts"])
            np.testing.assert_allclose(a["sums"], b["sums"], rtol=1e-12, atol=1e-12)


def test_group_by_fp32_value_counts_each_stored_value():
    """Rk-means step 1 groups by the values of a continuous attribute: one group per distinct
    stored FP32 value (its bit pattern), counted over the brute-force join."""
    rels = W.tiny_schema(7, max_rows=10, empty_ok=False)
    q = {"aggs": [[]], "groupby": [("x1", "float", None), ("k1", "value", None)], "filters": []}
    res = O.evaluate(rels, [q])[0]
    want = {}
    for r in materialise(rels):
        bits = int(np.array([r["x1"]], dtype=np.float32).view(np.uint32)[0])
        key = (bits, int(r["k1"]))
        want[key] = want.get(key, 0) + 1
    got = {(int(k[0]), int(k[1])): int(c) for k, c in zip(res["keys"], res["counts"])}
    assert got == want and len(got) > 1
