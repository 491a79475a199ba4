"""CPU oracle for batches of group-by aggregates over a natural join.

TEST INFRASTRUCTURE ONLY. Nothing in the engine imports this module: only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may call it. It shares no code with the CUDA path.

What it computes (Section 1 and Section 2 of the paper): every query of a batch is

    SELECT G, SUM(prod_i f_i(x)) ... FROM D WHERE cond GROUP BY G

over ``D``, the natural join of all relations (attributes with equal names are
equated). The oracle follows that definition literally and does none of the method's
optimisations (no views, no factorisation, no per-query roots):

1. ``natural_join`` materialises D as one row-index vector per relation, by hash-joining
   the relations one at a time on all attributes shared with the relations joined so far
   (duplicate keys give one joined tuple per combination; unmatched tuples drop out).
2. ``evaluate`` computes, per query, the filter mask (predicates compared on the stored
   FP32 / integer values), the group key of every joined tuple, each aggregate's product
   of factors in FP64 from the stored values, and sums them per group in FP64 in tuple
   order (``numpy.bincount``); COUNT is an INT64 count of joined tuples per group.
   It also returns, per aggregate and group, the sum of the absolute values of the terms,
   the scale against which the engine's rounding error is judged.
3. ``cart_variances`` derives the CART split variances (Section 3, decision trees):
   VARIANCE = SUM(y^2) - SUM(y)^2 / |T| for the left fragment (buckets 0..k) and the
   right fragment (the rest) of every threshold, in FP64.

Groups are returned in ascending lexicographic key order and only where COUNT > 0; an
ungrouped query always returns its single group, even when D is empty.
"""
from __future__ import annotations

import numpy as np

_OPS = {
    "le": np.less_equal, "lt": np.less, "ge": np.greater_equal, "gt": np.greater,
    "eq": np.equal, "ne": np.not_equal,
}


def _cols(R):
    return {c["attr"]: c for c in R["columns"]}


def natural_join(rels, order=None):
    """Row indices of the natural join of ``rels``: one int64 vector per relation.

    ``order`` is the sequence of relation positions to join (default: start from the
    first relation and repeatedly take the first remaining relation that shares an
    attribute with those joined so far). Each step joins on all shared attributes, so
    the result is the natural join whatever the order.
    """
    n = len(rels)
    if order is None:
        order = [0]
        joined_attrs = set(_cols(rels[0]))
        while len(order) < n:
            for i in range(n):
                if i not in order and joined_attrs & set(_cols(rels[i])):
                    order.append(i)
                    joined_attrs |= set(_cols(rels[i]))
                    break
            else:
                order.append(next(i for i in range(n) if i not in order))
                joined_attrs |= set(_cols(rels[order[-1]]))
    first = order[0]
    idx = {first: np.arange(rels[first]["nrows"], dtype=np.int64)}
    attr_home = {a: first for a in _cols(rels[first])}
    for i in order[1:]:
        R = rels[i]
        shared = [a for a in _cols(R) if a in attr_home]
        m = len(next(iter(idx.values())))
        if shared:
            # codes of both sides on the shared attributes, mixed radix with a radix that
            # exceeds every value seen on either side (so equal codes mean equal values)
            left = np.zeros(m, dtype=np.int64)
            right = np.zeros(R["nrows"], dtype=np.int64)
            for a in shared:
                home = attr_home[a]
                lv = _cols(rels[home])[a]["data"][idx[home]].astype(np.int64)
                rv = _cols(R)[a]["data"].astype(np.int64)
                radix = 1 + max(int(lv.max(initial=0)), int(rv.max(initial=0)))
                left = left * radix + lv
                right = right * radix + rv
            perm = np.argsort(right, kind="stable")
            rs = right[perm]
            lo = np.searchsorted(rs, left, side="left")
            hi = np.searchsorted(rs, left, side="right")
        else:
            perm = np.arange(R["nrows"], dtype=np.int64)
            lo = np.zeros(m, dtype=np.int64)
            hi = np.full(m, R["nrows"], dtype=np.int64)
        cnt = hi - lo
        rep = np.repeat(np.arange(m, dtype=np.int64), cnt)
        start = np.repeat(lo, cnt)
        offs = np.arange(len(rep), dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        for k in idx:
            idx[k] = idx[k][rep]
        idx[i] = perm[start + offs]
        for a in _cols(R):
            attr_home.setdefault(a, i)
    return [idx[i] for i in range(n)]


class JoinedData:
    """The materialised natural join: attribute values of every joined tuple."""

    def __init__(self, rels, order=None):
        self.rels = rels
        self.idx = natural_join(rels, order)
        self.size = len(self.idx[0]) if rels else 0
        self._home = {}
        for i, R in enumerate(rels):
            for c in R["columns"]:
                self._home.setdefault(c["attr"], (i, c))
        self._cache = {}

    def stored(self, attr):
        """Stored values (FP32 / integer, as loaded) of ``attr`` on every joined tuple."""
        i, c = self._home[attr]
        return c["data"][self.idx[i]]

    def f64(self, attr):
        if attr not in self._cache:
            self._cache[attr] = self.stored(attr).astype(np.float64)
        return self._cache[attr]


def _factor(J, f):
    attr, fn, p = f
    x = J.f64(attr)
    if fn == "id":
        return x
    if fn == "pow":
        out = np.ones_like(x)
        for _ in range(int(p)):
            out = out * x
        return out
    raise ValueError(f"unknown factor function {fn}")


def _group_code(J, g):
    attr, kind, thr = g
    v = J.stored(attr)
    if kind == "value":
        return v.astype(np.int64)
    if kind == "bucket":
        # bucket(x) = number of thresholds strictly below x (x == t lies in the <= side)
        t = np.asarray(thr, dtype=np.float32)
        return np.searchsorted(t, v.astype(np.float32), side="left").astype(np.int64)
    if kind == "float":
        # an FP32 value itself, as its 32-bit pattern (one group per distinct stored value)
        return v.astype(np.float32).view(np.uint32).astype(np.int64)
    raise ValueError(f"unknown group-by kind {kind}")


def evaluate_query(J, q):
    """One query over the materialised join ``J``; see the module docstring."""
    mask = np.ones(J.size, dtype=bool)
    for attr, op, t in q.get("filters", []):
        v = J.stored(attr)
        if v.dtype.kind == "f":
            mask &= _OPS[op](v, np.float32(t))
        else:
            mask &= _OPS[op](v.astype(np.float64), float(np.float32(t)))
    sel = np.nonzero(mask)[0]
    gb = q.get("groupby", [])
    if gb:
        codes = np.stack([_group_code(J, g)[sel] for g in gb], axis=1) if len(sel) else \
            np.zeros((0, len(gb)), dtype=np.int64)
        keys, inv = np.unique(codes, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        ng = len(keys)
    else:
        keys = np.zeros((1, 0), dtype=np.int64)
        inv = np.zeros(len(sel), dtype=np.int64)
        ng = 1
    counts = np.bincount(inv, minlength=ng).astype(np.int64)
    naggs = len(q["aggs"])
    sums = np.zeros((ng, naggs), dtype=np.float64)
    abs_sums = np.zeros((ng, naggs), dtype=np.float64)
    for j, agg in enumerate(q["aggs"]):
        term = np.ones(len(sel), dtype=np.float64)
        for f in agg:
            term = term * _factor(J, f)[sel]
        sums[:, j] = np.bincount(inv, weights=term, minlength=ng)
        abs_sums[:, j] = np.bincount(inv, weights=np.abs(term), minlength=ng)
    return {"keys": keys.astype(np.int64), "counts": counts, "sums": sums, "abs": abs_sums}


def evaluate(rels, queries, order=None):
    """All queries of a batch over the natural join of ``rels`` (FP64 sums, INT64 counts)."""
    J = JoinedData(rels, order)
    return [evaluate_query(J, q) for q in queries]


def cart_variances(result):
    """CART split variances from a bucketed query with aggregates COUNT, SUM(y), SUM(y^2)
    (Section 3): for every threshold k (between bucket k and k+1) the left fragment is
    buckets 0..k and the right fragment the remaining buckets; VARIANCE of a fragment T is
    SUM(y^2) - SUM(y)^2 / |T| (0 for an empty fragment). Returns (left, right) arrays over
    the thresholds of the bucket domain [0, nb) with nb = max bucket + 1 seen."""
    keys = result["keys"][:, 0]
    nb = int(keys.max()) + 1 if len(keys) else 1
    n = np.zeros(nb, dtype=np.int64)
    s = np.zeros(nb)
    s2 = np.zeros(nb)
    n[keys] = result["counts"]
    s[keys] = result["sums"][:, 1]
    s2[keys] = result["sums"][:, 2]

    def var(cnt, a, a2):
        out = np.zeros(len(cnt))
        nz = cnt > 0
        out[nz] = a2[nz] - a[nz] * a[nz] / cnt[nz]
        return out

    cn, cs, cs2 = np.cumsum(n), np.cumsum(s), np.cumsum(s2)
    left = var(cn[:-1], cs[:-1], cs2[:-1])
    right = var(cn[-1] - cn[:-1], cs[-1] - cs[:-1], cs2[-1] - cs2[:-1])
    return left, right


# ---------------------------------------------------------------------------------------
# Full-size evaluation: the join distributes over a partition of any one relation, so the
# batch over D is the sum of the batch over the joins of consecutive row chunks of the fact
# relation with the other relations (fixed 1M-tuple chunks, summed in chunk order, so the
# result does not depend on the number of processes).
# ---------------------------------------------------------------------------------------

CHUNK = 1_000_000


def _chunk_rels(rels, root, lo, hi):
    R = rels[root]
    part = dict(R, nrows=hi - lo, columns=[dict(c, data=c["data"][lo:hi]) for c in R["columns"]])
    return [part if i == root else X for i, X in enumerate(rels)]


def merge_results(queries, parts):
    """Sum per-chunk results (lists of per-query results, in chunk order) into one result
    per query: groups are the union of the chunks' groups, in ascending key order."""
    out = []
    for qi, q in enumerate(queries):
        rs = [p[qi] for p in parts]
        if not q.get("groupby"):
            counts = np.zeros(1, dtype=np.int64)
            sums = np.zeros((1, len(q["aggs"])))
            abs_ = np.zeros((1, len(q["aggs"])))
            for r in rs:
                counts += r["counts"]
                sums += r["sums"]
                abs_ += r["abs"]
            out.append({"keys": np.zeros((1, 0), dtype=np.int64), "counts": counts, "sums": sums, "abs": abs_})
            continue
        keys = np.concatenate([r["keys"] for r in rs], axis=0)
        uk, inv = np.unique(keys, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        ng = len(uk)
        counts = np.bincount(inv, weights=np.concatenate([r["counts"] for r in rs]).astype(np.float64),
                             minlength=ng)
        counts = np.rint(counts).astype(np.int64)
        S = np.concatenate([r["sums"] for r in rs], axis=0)
        A = np.concatenate([r["abs"] for r in rs], axis=0)
        sums = np.stack([np.bincount(inv, weights=S[:, j], minlength=ng) for j in range(S.shape[1])], axis=1) \
            if S.shape[1] else np.zeros((ng, 0))
        abs_ = np.stack([np.bincount(inv, weights=A[:, j], minlength=ng) for j in range(A.shape[1])], axis=1) \
            if A.shape[1] else np.zeros((ng, 0))
        keep = counts > 0
        out.append({"keys": uk[keep].astype(np.int64), "counts": counts[keep], "sums": sums[keep], "abs": abs_[keep]})
    return out


_W = {}  # worker state: the relations (fact columns attached from shared memory) and the batch


def _worker_init(spec, others, queries, root, chunk):
    from multiprocessing import shared_memory
    cols, shms = [], []
    for attr_meta, name, dtype, n in spec["cols"]:
        shm = shared_memory.SharedMemory(name=name)
        shms.append(shm)
        cols.append(dict(attr_meta, data=np.ndarray((n,), dtype=dtype, buffer=shm.buf)))
    fact = dict(spec["rel"], columns=cols)
    rels = list(others)
    rels.insert(root, fact)
    _W.update(rels=rels, queries=queries, root=root, shms=shms, chunk=chunk)


def _worker_chunk(i):
    rels, root, chunk = _W["rels"], _W["root"], _W["chunk"]
    n = rels[root]["nrows"]
    lo, hi = i * chunk, min(n, (i + 1) * chunk)
    return i, evaluate(_chunk_rels(rels, root, lo, hi), _W["queries"])


def evaluate_chunked(rels, queries, root=0, processes=1, chunk=CHUNK):
    """The batch over the natural join of ``rels``, evaluated over consecutive chunks of
    ``chunk`` rows of relation ``root`` and summed in chunk order (``merge_results``).
    With ``processes`` > 1 the chunks are spread over that many spawned processes that
    read the root relation's columns from shared memory (the sum order stays the chunk
    order). Returns (results, seconds)."""
    import time
    n = rels[root]["nrows"]
    nchunks = max(1, -(-n // chunk))
    t0 = time.perf_counter()
    if processes <= 1 or nchunks == 1:
        parts = [evaluate(_chunk_rels(rels, root, i * chunk, min(n, (i + 1) * chunk)), queries)
                 for i in range(nchunks)]
        return merge_results(queries, parts), time.perf_counter() - t0
    import multiprocessing as mp
    from multiprocessing import shared_memory
    R = rels[root]
    shms, spec_cols = [], []
    try:
        for c in R["columns"]:
            a = np.ascontiguousarray(c["data"])
            shm = shared_memory.SharedMemory(create=True, size=max(1, a.nbytes))
            shms.append(shm)
            np.ndarray(a.shape, dtype=a.dtype, buffer=shm.buf)[:] = a
            meta = {k: v for k, v in c.items() if k != "data"}
            spec_cols.append((meta, shm.name, a.dtype.str, len(a)))
        spec = {"rel": {k: v for k, v in R.items() if k != "columns"}, "cols": spec_cols}
        others = [X for i, X in enumerate(rels) if i != root]
        ctx = mp.get_context("spawn")
        with ctx.Pool(processes, initializer=_worker_init, initargs=(spec, others, queries, root, chunk)) as pool:
            parts = [None] * nchunks
            for i, res in pool.imap_unordered(_worker_chunk, range(nchunks)):
                parts[i] = res
    finally:
        for shm in shms:
            shm.close()
            shm.unlink()
    return merge_results(queries, parts), time.perf_counter() - t0


# ---------------------------------------------------------------------------------------
# Regression tree (Section 3, decision trees): the splits a CART learner chooses from the
# VARIANCE aggregates of every node, level by level.
# ---------------------------------------------------------------------------------------

def _tree_level_queries(target, features, thresholds, paths):
    qs = []
    for path in paths:
        for f in features:
            qs.append({"aggs": [[], [(target, "id", 1)], [(target, "pow", 2)]],
                       "groupby": [(f, "bucket", list(thresholds[f]))], "filters": list(path)})
    return qs


def best_split(results, nbuckets):
    """The split of one node from its per-feature bucketed (COUNT, SUM(y), SUM(y^2)) results:
    for feature f and threshold k (left = buckets 0..k, right = the rest), both sides
    non-empty, score = VARIANCE(left) + VARIANCE(right) with VARIANCE(T) = SUM(y^2) -
    SUM(y)^2 / |T|; the least score, ties to the lower feature, then the lower threshold.
    Returns (feature, k, score) or None."""
    best = None
    for f, (r, nb) in enumerate(zip(results, nbuckets)):
        n = np.zeros(nb)
        s = np.zeros(nb)
        s2 = np.zeros(nb)
        if len(r["keys"]):
            k = r["keys"][:, 0]
            n[k] = r["counts"]
            s[k] = r["sums"][:, 1]
            s2[k] = r["sums"][:, 2]
        tn, ts, ts2 = n.sum(), s.sum(), s2.sum()
        cn = cs = cs2 = 0.0
        for k in range(nb - 1):
            cn += n[k]
            cs += s[k]
            cs2 += s2[k]
            rn = tn - cn
            if cn <= 0 or rn <= 0:
                continue
            sc = (cs2 - cs * cs / cn) + ((ts2 - cs2) - (ts - cs) ** 2 / rn)
            if best is None or sc < best[2]:
                best = (f, k, sc)
    return best


def cart_tree(rels, target, features, thresholds, depth, processes=1):
    """Grow the tree of depth ``depth`` (levels 0 .. depth-1 choose splits) over the natural
    join of ``rels`` with the batches of ``_tree_level_queries`` evaluated by the oracle
    (whole-join evaluation, chunked over ``processes``). Nodes in heap order: dicts with
    active, feature (-1: no valid split), threshold, score, count, sum_y, sum_y2."""
    nn = (1 << depth) - 1
    nodes = [{"active": 0, "feature": -1, "threshold": 0.0, "score": 0.0, "count": 0, "sum_y": 0.0, "sum_y2": 0.0}
             for _ in range(nn)]
    paths = [[] for _ in range(nn)]
    nodes[0]["active"] = 1
    nb = [len(thresholds[f]) + 1 for f in features]
    for lev in range(depth):
        act = [v for v in range((1 << lev) - 1, (1 << (lev + 1)) - 1) if nodes[v]["active"]]
        if not act:
            continue
        qs = _tree_level_queries(target, features, thresholds, [paths[v] for v in act])
        res, _ = evaluate_chunked(rels, qs, root=0, processes=processes)
        for i, v in enumerate(act):
            rs = res[i * len(features):(i + 1) * len(features)]
            cnt = sum(int(x) for x in rs[0]["counts"])
            nodes[v].update(count=cnt, sum_y=float(rs[0]["sums"][:, 1].sum()), sum_y2=float(rs[0]["sums"][:, 2].sum()))
            b = best_split(rs, nb)
            if b is None:
                continue
            f, k, sc = b
            t = float(np.float32(thresholds[features[f]][k]))
            nodes[v].update(feature=f, threshold=t, score=float(sc))
            if 2 * v + 2 < nn:
                for c, op in ((1, "le"), (2, "gt")):
                    paths[2 * v + c] = paths[v] + [(features[f], op, t)]
                    nodes[2 * v + c]["active"] = 1
    return nodes


# ---------------------------------------------------------------------------------------
# Ridge regression from the aggregates (Section 3, linear regression)
# ---------------------------------------------------------------------------------------

def ridge_system(result, query, target, features):
    """(A, b, syy) of the ridge objective J(theta) = 1/(2|D|) SUM_D (theta^T x - y)^2 +
    lambda/2 |theta|^2 without lambda: A = SUM x x^T / |D|, b = SUM x y / |D|, syy = SUM y^2 /
    |D| with x = (1, features), read from the ungrouped query's aggregates by their factors."""
    def key(agg):
        k = {}
        for a, fn, p in agg:
            k[a] = k.get(a, 0) + (int(p) if fn == "pow" else 1)
        return tuple(sorted(k.items()))
    pos = {key(a): j for j, a in enumerate(query["aggs"])}
    n = float(result["counts"][0])
    z = [None] + list(features) + [target]
    w = len(z)
    M = np.zeros((w, w))
    for i in range(w):
        for j in range(w):
            if i == 0 and j == 0:
                M[i, j] = n
                continue
            k = {}
            for a in (z[i], z[j]):
                if a is not None:
                    k[a] = k.get(a, 0) + 1
            M[i, j] = result["sums"][0, pos[tuple(sorted(k.items()))]]
    M /= n
    m = w - 1
    return M[:m, :m], M[:m, m], M[m, m]


def ridge_closed_form(A, b, lam):
    """theta with grad J = (A + lam I) theta - b = 0."""
    return np.linalg.solve(A + lam * np.eye(len(b)), b)


def ridge_bgd(A, b, lam, iters, step):
    """Batch gradient descent on J from theta = 0: theta <- theta - step * grad J(theta)."""
    th = np.zeros(len(b))
    for _ in range(iters):
        th = th - step * ((A + lam * np.eye(len(b))) @ th - b)
    return th


def ridge_objective(A, b, syy, lam, th):
    return 0.5 * (th @ A @ th - 2 * th @ b + syy) + 0.5 * lam * th @ th
