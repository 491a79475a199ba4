"""Seeded synthetic relations and aggregate batches shaped like the paper's workloads.

The paper learns its models over two multi-relational datasets, Retailer (84M fact
tuples) and Favorita (120M fact tuples) (Section 1), with the Favorita schema drawn in
Fig. 2. Neither dataset is available here, so this module generates stand-ins of the
same shape: the same relations, join keys, key domains, feature counts and categorical
domains, with values from a seeded ``numpy`` generator.

This module only *describes inputs*: relations (columns with a role and a domain) and
query batches (aggregates, group-by attributes, filters). It performs no join and no
aggregation, so it can feed both the CUDA engine and the CPU oracle without giving either
one the other's arithmetic.

Vocabulary (shared by the binding and the oracle):

* relation: ``{"name", "nrows", "columns": [column, ...]}``
* column:   ``{"attr", "data" (numpy array), "role" ("key"|"cat"|"cont"), "domain"}``;
  ``key`` columns are join attributes (int32 values in ``[0, domain)``), ``cat`` columns
  are categorical (int32 in ``[0, domain)``), ``cont`` columns are float32 (or uint8 0/1).
  Attributes with equal names join (natural join, Section 2).
* query:    ``{"aggs": [[factor, ...], ...], "groupby": [group, ...], "filters": [pred, ...]}``
  where an aggregate is ``SUM(prod factors)`` (an empty factor list is ``SUM(1)``),
  ``factor = (attr, "id"|"pow", p)``, ``group = (attr, "value"|"bucket", thresholds)``,
  ``pred = (attr, "le"|"lt"|"ge"|"gt"|"eq"|"ne", t)`` (conjunctive, Section 3 CART).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

KEY, CAT, CONT = "key", "cat", "cont"


def column(attr, data, role, domain=0):
    return {"attr": attr, "data": np.ascontiguousarray(data), "role": role, "domain": int(domain)}


def relation(name, cols):
    n = len(cols[0]["data"])
    for c in cols:
        if len(c["data"]) != n:
            raise ValueError(f"column {c['attr']} of {name} has {len(c['data'])} rows, expected {n}")
    return {"name": name, "nrows": n, "columns": cols}


def _rng(seed, salt):
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(salt)]))


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def _i32(x):
    return np.asarray(x, dtype=np.int32)


# ---------------------------------------------------------------------------------------
# Batch builders (Section 3: ridge regression aggregates; CART aggregates)
# ---------------------------------------------------------------------------------------

def ridge_batch(conts, cats):
    """Ridge-regression batch over the continuous attributes ``conts`` (Section 3, LR).

    One ungrouped query holds COUNT, SUM(x_i) and SUM(x_i * x_j) for i <= j (the
    non-centred covariance matrix Sigma, with the intercept column x_1 = 1 giving the
    COUNT and the SUM(x_i) entries). Categorical attributes are one-hot encoded as
    group-by attributes: for each categorical X_j a query ``X_j, COUNT, SUM(x_k) GROUP BY
    X_j`` (cat x cont entries), and for each pair a query ``X_j, X_k, SUM(1) GROUP BY X_j, X_k``
    (cat x cat entries).
    """
    aggs = [[]]
    aggs += [[(x, "id", 1)] for x in conts]
    for i, a in enumerate(conts):
        for b in conts[i:]:
            aggs.append([(a, "pow", 2)] if a == b else [(a, "id", 1), (b, "id", 1)])
    queries = [{"aggs": aggs, "groupby": [], "filters": []}]
    for c in cats:
        queries.append({"aggs": [[]] + [[(x, "id", 1)] for x in conts],
                        "groupby": [(c, "value", None)], "filters": []})
    for c1, c2 in itertools.combinations(cats, 2):
        queries.append({"aggs": [[]], "groupby": [(c1, "value", None), (c2, "value", None)],
                        "filters": []})
    return queries


# ---------------------------------------------------------------------------------------
# Config 0: star join, 200k fact rows, two dimensions
# ---------------------------------------------------------------------------------------

def star_schema(n_fact=200_000, seed=0, n_d1=1000, n_d2=500):
    """Fact F(a, b, y, f1, f2) with FKs a -> D1 and b -> D2; D1(a, x1..x3, c1/16); D2(b, z1, z2, c2/8)."""
    r, rd = _rng(seed, 0), _rng(seed, 100)
    F = relation("F", [
        column("a", _i32(r.integers(0, n_d1, n_fact)), KEY, n_d1),
        column("b", _i32(r.integers(0, n_d2, n_fact)), KEY, n_d2),
        column("y", _f32(r.standard_normal(n_fact)), CONT),
        column("f1", _f32(r.standard_normal(n_fact)), CONT),
        column("f2", _f32(r.standard_normal(n_fact)), CONT),
    ])
    r = rd
    D1 = relation("D1", [
        column("a", _i32(np.arange(n_d1)), KEY, n_d1),
        column("x1", _f32(r.random(n_d1)), CONT),
        column("x2", _f32(r.random(n_d1)), CONT),
        column("x3", _f32(r.random(n_d1)), CONT),
        column("c1", _i32(r.integers(0, 16, n_d1)), CAT, 16),
    ])
    D2 = relation("D2", [
        column("b", _i32(np.arange(n_d2)), KEY, n_d2),
        column("z1", _f32(r.standard_normal(n_d2)), CONT),
        column("z2", _f32(r.standard_normal(n_d2)), CONT),
        column("c2", _i32(r.integers(0, 8, n_d2)), CAT, 8),
    ])
    return [F, D1, D2]


STAR_CONTS = ["y", "f1", "f2", "x1", "x2", "x3", "z1", "z2"]
STAR_CATS = ["c1", "c2"]


def star_batch():
    return ridge_batch(STAR_CONTS, STAR_CATS)


# ---------------------------------------------------------------------------------------
# Config 1: Retailer-shaped snowflake (Inventory, Item, Location -> Census, Weather)
# ---------------------------------------------------------------------------------------

N_LOCN, N_DATE, N_ITEM, N_ZIP = 1300, 124, 3700, 1300
N_WEATHER = 160_000


def retailer_schema(n_fact=84_000_000, seed=0):
    """Retailer-shaped 5-relation snowflake.

    Inventory(locn, date, item, y) with y lognormal; Item(item, i1..i4, cat_item/50);
    Location(locn, zip, l1..l10, cat_locn/24) with zip -> Census(zip, c1..c14, cat_zip/12);
    Weather(locn, date, w1..w8) holding 160,000 of the 161,200 (locn, date) pairs, so fact
    tuples whose pair is absent drop out of the natural join.
    """
    r, rd = _rng(seed, 1), _rng(seed, 101)
    F = relation("Inventory", [
        column("locn", _i32(r.integers(0, N_LOCN, n_fact)), KEY, N_LOCN),
        column("date", _i32(r.integers(0, N_DATE, n_fact)), KEY, N_DATE),
        column("item", _i32(r.integers(0, N_ITEM, n_fact)), KEY, N_ITEM),
        column("y", _f32(np.exp(r.standard_normal(n_fact, dtype=np.float32))), CONT),
    ])
    r = rd
    item = relation("Item", [column("item", _i32(np.arange(N_ITEM)), KEY, N_ITEM)]
                    + [column(f"i{k}", _f32(r.standard_normal(N_ITEM)), CONT) for k in range(1, 5)]
                    + [column("cat_item", _i32(r.integers(0, 50, N_ITEM)), CAT, 50)])
    loc = relation("Location", [column("locn", _i32(np.arange(N_LOCN)), KEY, N_LOCN),
                                column("zip", _i32(r.integers(0, N_ZIP, N_LOCN)), KEY, N_ZIP)]
                   + [column(f"l{k}", _f32(r.standard_normal(N_LOCN)), CONT) for k in range(1, 11)]
                   + [column("cat_locn", _i32(r.integers(0, 24, N_LOCN)), CAT, 24)])
    census = relation("Census", [column("zip", _i32(np.arange(N_ZIP)), KEY, N_ZIP)]
                      + [column(f"c{k}", _f32(r.standard_normal(N_ZIP)), CONT) for k in range(1, 15)]
                      + [column("cat_zip", _i32(r.integers(0, 12, N_ZIP)), CAT, 12)])
    pairs = r.choice(N_LOCN * N_DATE, N_WEATHER, replace=False)
    weather = relation("Weather", [column("locn", _i32(pairs // N_DATE), KEY, N_LOCN),
                                   column("date", _i32(pairs % N_DATE), KEY, N_DATE)]
                       + [column(f"w{k}", _f32(r.standard_normal(N_WEATHER)), CONT) for k in range(1, 9)])
    return [F, item, loc, census, weather]


RETAILER_CONTS = (["y"] + [f"i{k}" for k in range(1, 5)] + [f"l{k}" for k in range(1, 11)]
                  + [f"c{k}" for k in range(1, 15)] + [f"w{k}" for k in range(1, 9)])
RETAILER_CATS = ["cat_locn", "cat_zip", "cat_item"]


def retailer_batch():
    return ridge_batch(RETAILER_CONTS, RETAILER_CATS)


# ---------------------------------------------------------------------------------------
# Config 2: Favorita-shaped schema of Fig. 2 (Sales, Transactions, StoRes, Oil, Holidays, Items)
# ---------------------------------------------------------------------------------------

N_FDATE, N_STORE, N_FITEM = 1684, 54, 4100
N_TRANS = 84_000


def favorita_schema(n_fact=120_000_000, seed=0):
    """Favorita-shaped 6-relation schema (Fig. 2).

    Sales(date, store, item, units, promo); Transactions(date, store, txns) holding 84,000
    of the 90,936 (date, store) pairs; StoRes(store, city/22, state/16, stype/5,
    cluster/17); Oil(date, price); Holidays(date, htype/6, locale/3, transferred/2);
    Items(item, family/33, class/337, perishable/2). ``promo`` is a 0/1 uint8 column with
    P(1) = 0.1.
    """
    r, rd = _rng(seed, 2), _rng(seed, 102)
    S = relation("Sales", [
        column("date", _i32(r.integers(0, N_FDATE, n_fact)), KEY, N_FDATE),
        column("store", _i32(r.integers(0, N_STORE, n_fact)), KEY, N_STORE),
        column("item", _i32(r.integers(0, N_FITEM, n_fact)), KEY, N_FITEM),
        column("units", _f32(np.exp(r.standard_normal(n_fact, dtype=np.float32))), CONT),
        column("promo", (r.random(n_fact, dtype=np.float32) < 0.1).astype(np.uint8), CONT),
    ])
    r = rd
    pairs = r.choice(N_FDATE * N_STORE, N_TRANS, replace=False)
    T = relation("Transactions", [column("date", _i32(pairs // N_STORE), KEY, N_FDATE),
                                  column("store", _i32(pairs % N_STORE), KEY, N_STORE),
                                  column("txns", _f32(np.exp(r.standard_normal(N_TRANS))), CONT)])
    R = relation("StoRes", [column("store", _i32(np.arange(N_STORE)), KEY, N_STORE),
                            column("city", _i32(r.integers(0, 22, N_STORE)), CAT, 22),
                            column("state", _i32(r.integers(0, 16, N_STORE)), CAT, 16),
                            column("stype", _i32(r.integers(0, 5, N_STORE)), CAT, 5),
                            column("cluster", _i32(r.integers(0, 17, N_STORE)), CAT, 17)])
    O = relation("Oil", [column("date", _i32(np.arange(N_FDATE)), KEY, N_FDATE),
                         column("price", _f32(r.standard_normal(N_FDATE)), CONT)])
    H = relation("Holidays", [column("date", _i32(np.arange(N_FDATE)), KEY, N_FDATE),
                              column("htype", _i32(r.integers(0, 6, N_FDATE)), CAT, 6),
                              column("locale", _i32(r.integers(0, 3, N_FDATE)), CAT, 3),
                              column("transferred", _i32(r.integers(0, 2, N_FDATE)), CAT, 2)])
    I = relation("Items", [column("item", _i32(np.arange(N_FITEM)), KEY, N_FITEM),
                           column("family", _i32(r.integers(0, 33, N_FITEM)), CAT, 33),
                           column("class", _i32(r.integers(0, 337, N_FITEM)), CAT, 337),
                           column("perishable", _i32(r.integers(0, 2, N_FITEM)), CAT, 2)])
    return [S, T, R, O, H, I]


FAVORITA_CONTS = ["units", "promo", "txns", "price"]
FAVORITA_CATS = ["family", "class", "perishable", "city", "state", "stype", "cluster",
                 "htype", "locale", "transferred"]
# Join tree of Fig. 2 (child -> parent)
FAVORITA_TREE = {"Transactions": "Sales", "StoRes": "Transactions", "Oil": "Transactions",
                 "Items": "Sales", "Holidays": "Sales"}


def favorita_batch():
    return ridge_batch(FAVORITA_CONTS, FAVORITA_CATS)


def favorita_example_queries():
    """Q1-Q3 of Section 2: Q1 = SUM(units); Q2 = SUM(g(item) * h(date)) GROUP BY store;
    Q3 = SUM(units * price) GROUP BY class. g and h are taken as the identity on the key."""
    return [
        {"aggs": [[("units", "id", 1)]], "groupby": [], "filters": []},
        {"aggs": [[("item", "id", 1), ("date", "id", 1)]], "groupby": [("store", "value", None)],
         "filters": []},
        {"aggs": [[("units", "id", 1), ("price", "id", 1)]], "groupby": [("class", "value", None)],
         "filters": []},
    ]


# ---------------------------------------------------------------------------------------
# Config 3: one decision-tree level on the Retailer-shaped schema (Section 3, CART)
# ---------------------------------------------------------------------------------------

N_BUCKET_THRESH = 19


def _feature_values(rels, attr):
    for R in rels:
        for c in R["columns"]:
            if c["attr"] == attr and c["role"] == CONT:
                return c["data"]
    raise KeyError(attr)


def bucket_thresholds(rels, conts, seed=0, max_sample=1_000_000):
    """19 interior thresholds per feature: the FP32 equi-depth quantiles k/20 of the
    feature over its base relation (a seeded sample of at most ``max_sample`` values)."""
    r = _rng(seed, 3)
    out = {}
    for a in conts:
        v = _feature_values(rels, a)
        if len(v) > max_sample:
            v = v[r.integers(0, len(v), max_sample)]
        q = np.quantile(v.astype(np.float64), np.arange(1, N_BUCKET_THRESH + 1) / (N_BUCKET_THRESH + 1))
        out[a] = np.unique(_f32(q))
    return out


def _leaf_filters(splits):
    """Conjunctive filters of the 8 leaves of a depth-4 binary tree whose 7 internal
    nodes (heap order) carry splits (attr, t): left branch attr <= t, right attr > t."""
    leaves = []
    for leaf in range(8):
        preds, node = [], 0
        for depth in range(3):
            bit = (leaf >> (2 - depth)) & 1
            a, t = splits[node]
            preds.append((a, "gt" if bit else "le", float(t)))
            node = 2 * node + 1 + bit
        leaves.append(preds)
    return leaves


def dt_level_batch(rels, conts=RETAILER_CONTS, target="y", seed=0, lo=0.01, hi=0.40,
                   sample_rows=200_000):
    """The 8 leaves of a depth-4 regression tree, each with its conjunctive filter of 3
    threshold predicates, and for every feature its 20 buckets: COUNT, SUM(y), SUM(y^2)
    per bucket per node (Section 3, CART; the VARIANCE of a split follows from them).

    The 7 splits are drawn with the seed from the non-target features and their bucket
    thresholds and redrawn until every leaf holds between ``lo`` and ``hi`` of a sample
    of the fact relation (fact rows of the sample are resolved against unique-key
    dimensions by direct indexing; rows with unresolved keys are ignored).
    Returns (queries, splits, thresholds).
    """
    r = _rng(seed, 4)
    thr = bucket_thresholds(rels, conts, seed)
    feats = [a for a in conts if a != target]
    vals = _sample_feature_rows(rels, feats, sample_rows, r)
    for _ in range(10_000):
        splits = []
        for _n in range(7):
            a = feats[int(r.integers(0, len(feats)))]
            t = thr[a][int(r.integers(0, len(thr[a])))]
            splits.append((a, np.float32(t)))
        leaf = np.zeros(len(next(iter(vals.values()))), dtype=np.int64)
        node = np.zeros_like(leaf)
        for depth in range(3):
            a_of = np.array([splits[k][0] for k in range(7)])
            t_of = np.array([splits[k][1] for k in range(7)], dtype=np.float32)
            go_right = np.zeros_like(leaf, dtype=bool)
            for k in range(7):
                m = node == k
                if m.any():
                    go_right[m] = vals[a_of[k]][m] > t_of[k]
            leaf = leaf * 2 + go_right
            node = 2 * node + 1 + go_right
        frac = np.bincount(leaf, minlength=8) / len(leaf)
        if frac.min() >= lo and frac.max() <= hi:
            break
    else:
        raise RuntimeError("no tree with balanced leaves found")
    filters = _leaf_filters(splits)
    queries = []
    for preds in filters:
        for a in conts:
            queries.append({"aggs": [[], [(target, "id", 1)], [(target, "pow", 2)]],
                            "groupby": [(a, "bucket", thr[a])], "filters": list(preds)})
    return queries, splits, thr


def _sample_feature_rows(rels, feats, n, r):
    """Feature values for a sample of fact rows of the Retailer-shaped schema, resolved
    through its unique-key dimensions by direct indexing (input-selection helper)."""
    F, item, loc, census, weather = rels
    fc = {c["attr"]: c["data"] for c in F["columns"]}
    idx = r.integers(0, F["nrows"], min(n, F["nrows"]))
    locn, date, it = fc["locn"][idx], fc["date"][idx], fc["item"][idx]
    wpos = np.full(N_LOCN * N_DATE, -1, dtype=np.int64)
    wc = {c["attr"]: c["data"] for c in weather["columns"]}
    wpos[wc["locn"].astype(np.int64) * N_DATE + wc["date"]] = np.arange(weather["nrows"])
    wrow = wpos[locn.astype(np.int64) * N_DATE + date]
    keep = wrow >= 0
    lc = {c["attr"]: c["data"] for c in loc["columns"]}
    cc = {c["attr"]: c["data"] for c in census["columns"]}
    ic = {c["attr"]: c["data"] for c in item["columns"]}
    zipv = lc["zip"][locn]
    out = {}
    for a in feats:
        if a in ic:
            v = ic[a][it]
        elif a in lc:
            v = lc[a][locn]
        elif a in cc:
            v = cc[a][zipv]
        elif a in wc:
            v = wc[a][np.maximum(wrow, 0)]
        else:
            v = fc[a][idx]
        out[a] = v[keep]
    return out


# ---------------------------------------------------------------------------------------
# Config 4: random acyclic (snowflake) schemas for the learned planner
# ---------------------------------------------------------------------------------------

def random_snowflake(seed, n_fact=None, fact_range=(1e5, 5e7), rel_range=(3, 8),
                     dom_range=(10, 1e5), feat_range=(2, 12)):
    """A seeded random snowflake: a fact relation F and 2..7 dimension relations, each
    with a unique key (its key domain = its row count) referenced by an FK of its parent
    (uniform, or Zipf(1.1) with probability 1/2). Every relation carries 2..12 float32
    features; every dimension one categorical of 2..16 values. Returns (rels, parent map,
    conts, cats)."""
    r = _rng(seed, 5)
    n_rel = int(r.integers(rel_range[0], rel_range[1] + 1))
    if n_fact is None:
        n_fact = int(round(math.exp(r.uniform(math.log(fact_range[0]), math.log(fact_range[1])))))
    parents = {}
    names = ["F"] + [f"R{k}" for k in range(1, n_rel)]
    doms = {}
    for k in range(1, n_rel):
        parents[names[k]] = names[int(r.integers(0, k))]
        doms[names[k]] = int(round(math.exp(r.uniform(math.log(dom_range[0]), math.log(dom_range[1])))))
    nrows = {"F": n_fact, **doms}
    cols = {n: [] for n in names}
    for child, par in parents.items():
        key = f"k_{child}"
        d = doms[child]
        if r.random() < 0.5:
            fk = r.integers(0, d, nrows[par])
        else:
            fk = _zipf_keys(r, d, nrows[par], 1.1)
        cols[par].append(column(key, _i32(fk), KEY, d))
        cols[child].insert(0, column(key, _i32(r.permutation(d)), KEY, d))
    conts, cats = [], []
    for n in names:
        nf = int(r.integers(feat_range[0], feat_range[1] + 1))
        for j in range(nf):
            a = f"{n}_x{j}"
            cols[n].append(column(a, _f32(r.standard_normal(nrows[n])), CONT))
            conts.append(a)
        if n != "F":
            g = int(r.integers(2, 17))
            a = f"{n}_g"
            cols[n].append(column(a, _i32(r.integers(0, g, nrows[n])), CAT, g))
            cats.append(a)
    rels = [relation(n, cols[n]) for n in names]
    return rels, parents, conts, cats


def _zipf_keys(r, d, n, s):
    w = 1.0 / np.arange(1, d + 1) ** s
    w /= w.sum()
    perm = r.permutation(d)
    return perm[r.choice(d, n, p=w)]


def scaled(rels, fact_rows, seed=0, fact_name=None):
    """The first ``fact_rows`` rows of the fact relation (the first relation or
    ``fact_name``), other relations unchanged: a smaller instance of the same workload."""
    out = []
    for i, R in enumerate(rels):
        if (fact_name is None and i == 0) or R["name"] == fact_name:
            out.append(relation(R["name"], [dict(c, data=c["data"][:fact_rows]) for c in R["columns"]]))
        else:
            out.append(R)
    return out


# ---------------------------------------------------------------------------------------
# Tiny random schemas (duplicate and dangling keys) for brute-force checks
# ---------------------------------------------------------------------------------------

def tiny_schema(seed, max_rows=12, kdom=4, shared3=False, empty_ok=True, fd=False):
    """A tiny acyclic schema with duplicate and dangling join keys.

    R0(k1, k2, x0, g0/3) joins R1(k1, x1, g1/2) on k1 and R2(k2, k3, x2) on k2; R2 joins
    R3(k3, x3, g3/3) on k3. With ``shared3`` a fifth relation R4(k1, k2, x4) shares both
    of R0's keys (k1 then appears in three relations). Keys are drawn from ``[0, kdom)``
    with repetition, so some keys repeat and some have no partner. With ``fd`` the
    relations holding categoricals (R1, R3) get distinct keys, so their categoricals are
    determined by their join key (the other relations keep repeated keys).
    """
    r = _rng(seed, 6)

    def n():
        lo = 0 if empty_ok and r.random() < 0.05 else 1
        return int(r.integers(lo, max_rows + 1))

    def keys(m, d=kdom):
        return _i32(r.integers(0, d, m))

    def vals(m):
        return _f32(np.round(r.standard_normal(m) * 4) / 4)

    m0, m1, m2, m3 = n(), n(), n(), n()
    if fd:
        m1, m3 = min(m1, kdom - 1), min(m3, kdom - 1)

    def ukeys(m):
        return _i32(r.permutation(kdom)[:m]) if fd else keys(m)

    rels = [
        relation("R0", [column("k1", keys(m0), KEY, kdom), column("k2", keys(m0), KEY, kdom),
                        column("x0", vals(m0), CONT), column("g0", keys(m0, 3), CAT, 3)]),
        relation("R1", [column("k1", ukeys(m1), KEY, kdom), column("x1", vals(m1), CONT),
                        column("g1", keys(m1, 2), CAT, 2)]),
        relation("R2", [column("k2", keys(m2), KEY, kdom), column("k3", keys(m2), KEY, kdom),
                        column("x2", vals(m2), CONT)]),
        relation("R3", [column("k3", ukeys(m3), KEY, kdom), column("x3", vals(m3), CONT),
                        column("g3", keys(m3, 3), CAT, 3)]),
    ]
    if shared3:
        m4 = n()
        rels.append(relation("R4", [column("k1", keys(m4), KEY, kdom), column("k2", keys(m4), KEY, kdom),
                                    column("x4", vals(m4), CONT)]))
    return rels


def tiny_queries(seed, rels, nq=6, group_attrs=None, bucket_attrs=None):
    """Random queries over a tiny schema: products of 0..3 factors (with powers),
    0..2 group-by attributes (values or buckets), 0..2 filter predicates. Group-by
    attributes are drawn from ``group_attrs`` / ``bucket_attrs`` when given."""
    r = _rng(seed, 7)
    conts = [c["attr"] for R in rels for c in R["columns"] if c["role"] == CONT]
    cats = sorted({c["attr"] for R in rels for c in R["columns"] if c["role"] in (CAT, KEY)})
    gcats = cats if group_attrs is None else list(group_attrs)
    gconts = conts if bucket_attrs is None else list(bucket_attrs)
    ops = ["le", "lt", "ge", "gt", "eq", "ne"]
    qs = []
    for _ in range(nq):
        aggs = [[]]
        for _a in range(int(r.integers(1, 5))):
            k = int(r.integers(0, 4))
            aggs.append([(conts[int(r.integers(0, len(conts)))], "pow" if r.random() < 0.3 else "id",
                          int(r.integers(2, 4))) for _f in range(k)])
            aggs[-1] = [(a, fn, p if fn == "pow" else 1) for a, fn, p in aggs[-1]]
        gb = []
        for _g in range(int(r.integers(0, 3))):
            if r.random() < 0.3 and gconts:
                a = gconts[int(r.integers(0, len(gconts)))]
                if a not in [g[0] for g in gb]:
                    gb.append((a, "bucket", np.array([-1.0, 0.0, 0.5], dtype=np.float32)))
            elif gcats:
                a = gcats[int(r.integers(0, len(gcats)))]
                if a not in [g[0] for g in gb]:
                    gb.append((a, "value", None))
        flt = []
        for _p in range(int(r.integers(0, 3))):
            a = (conts + cats)[int(r.integers(0, len(conts) + len(cats)))]
            flt.append((a, ops[int(r.integers(0, 6))], float(np.float32(r.choice([-0.5, 0.0, 0.25, 1.0, 2.0])))))
        qs.append({"aggs": aggs, "groupby": gb, "filters": flt})
    return qs
