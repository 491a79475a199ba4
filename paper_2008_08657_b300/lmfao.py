"""Thin ctypes binding of the C ABI in ``include/lmfao.h`` (argument marshalling only).

Every step of the evaluation runs in the CUDA kernels of ``liblmfao.so``; this module
converts Python descriptions of relations and queries (the vocabulary of
``workloads.py``) into the C structs and back. Loading fails loudly when the library is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblmfao.so")

OK, ERR_ARG, ERR_DTYPE, ERR_KEY_RANGE, ERR_CYCLIC, ERR_NOT_PLANNED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, \
    ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
I32, F32, U8 = 0, 1, 2
KEY, CAT, CONT = 0, 1, 2
HOST, DEVICE, ADOPT_DEVICE = 0, 1, 2
FN_ID, FN_POW = 0, 1
GB_VALUE, GB_BUCKET = 0, 1
OPS = {"le": 0, "lt": 1, "ge": 2, "gt": 3, "eq": 4, "ne": 5}
PRECISION = {"fp64": 0, "fp32": 1, "split_bf16": 2}
PLANNER = {"heuristic": 0, "exhaustive": 1, "learned": 2, "forced": 3}
MODE = {"auto": 0, "factorised": 1, "per_tuple": 2, "generic": 3}
ROLE = {"key": KEY, "cat": CAT, "cont": CONT}

# The C entry points of include/lmfao.h (checked by the tests against the header).
ENTRY_POINTS = [
    "lmfao_create", "lmfao_destroy", "lmfao_last_error", "lmfao_load_relation", "lmfao_add_batch",
    "lmfao_clear_batch", "lmfao_plan", "lmfao_run", "lmfao_fetch", "lmfao_result_device",
    "lmfao_describe_plan", "lmfao_cart_variances", "lmfao_kernel_times", "lmfao_kernel_name",
    "lmfao_set_profiling", "lmfao_cart_variances_noalloc", "lmfao_mlp_param_count", "lmfao_mlp_forward",
    "lmfao_mlp_loss", "lmfao_mlp_backward", "lmfao_mlp_adam", "lmfao_plan_candidates", "lmfao_result_state",
    "lmfao_cart_tree", "lmfao_ridge_fit", "lmfao_group_count",
]
COST_MODEL_PATH = os.path.join(_HERE, "cost_model.txt")


class Column(C.Structure):
    _fields_ = [("attr", C.c_char_p), ("dtype", C.c_int32), ("role", C.c_int32), ("domain", C.c_int64),
                ("data", C.c_void_p)]


class Factor(C.Structure):
    _fields_ = [("attr", C.c_char_p), ("fn", C.c_int32), ("param", C.c_int32)]


class Aggregate(C.Structure):
    _fields_ = [("factors", C.POINTER(Factor)), ("nfactors", C.c_int32)]


class GroupBy(C.Structure):
    _fields_ = [("attr", C.c_char_p), ("kind", C.c_int32), ("nthresholds", C.c_int32),
                ("thresholds", C.POINTER(C.c_float))]


class Predicate(C.Structure):
    _fields_ = [("attr", C.c_char_p), ("op", C.c_int32), ("t", C.c_float)]


class PlanOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("planner", C.c_int32), ("root_rel", C.c_int32),
                ("segment_rel", C.c_int32), ("mode", C.c_int32), ("autotune", C.c_int32),
                ("join_parent", C.POINTER(C.c_int32)), ("query_root", C.POINTER(C.c_int32)),
                ("cost_model", C.c_char_p), ("combine", C.c_int32), ("learned_topk", C.c_int32)]


class PlanInfo(C.Structure):
    _fields_ = [("root_rel", C.c_int32), ("segment_rel", C.c_int32), ("n_segments", C.c_int64),
                ("n_views", C.c_int32), ("n_groups", C.c_int32), ("n_kernels", C.c_int32),
                ("mode", C.c_int32), ("predicted_ms", C.c_double), ("plan_ms", C.c_double),
                ("reorg_ms", C.c_double), ("reorg_reused", C.c_int32), ("n_roots", C.c_int32)]


class CartNode(C.Structure):
    _fields_ = [("active", C.c_int32), ("feature", C.c_int32), ("threshold", C.c_float), ("score", C.c_double),
                ("count", C.c_int64), ("sum_y", C.c_double), ("sum_y2", C.c_double)]


class Result(C.Structure):
    _fields_ = [("ngroups", C.c_int64), ("ngroupby", C.c_int32), ("naggs", C.c_int32),
                ("group_keys", C.POINTER(C.c_int32)), ("counts", C.POINTER(C.c_int64)),
                ("sums", C.POINTER(C.c_double))]


class LmfaoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lmfao error {code}: {msg}")
        self.code = code


_lib = None


def library():
    """The loaded ``liblmfao.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2008_08657_b300/build.py (there is no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sig = {
            "lmfao_create": (C.c_int, [C.POINTER(P), C.c_int]),
            "lmfao_destroy": (C.c_int, [P]),
            "lmfao_last_error": (C.c_char_p, [P]),
            "lmfao_load_relation": (C.c_int, [P, C.c_char_p, C.c_int64, C.POINTER(Column), C.c_int, C.c_uint32,
                                              C.POINTER(C.c_int)]),
            "lmfao_add_batch": (C.c_int, [P, C.POINTER(Aggregate), C.c_int, C.POINTER(GroupBy), C.c_int,
                                          C.POINTER(Predicate), C.c_int, C.POINTER(C.c_int)]),
            "lmfao_clear_batch": (C.c_int, [P]),
            "lmfao_plan": (C.c_int, [P, C.POINTER(PlanOpts), C.POINTER(PlanInfo)]),
            "lmfao_run": (C.c_int, [P, P]),
            "lmfao_fetch": (C.c_int, [P, C.c_int, C.POINTER(Result)]),
            "lmfao_result_device": (C.c_int, [P, C.c_int, P, P, C.POINTER(C.c_int64), P]),
            "lmfao_result_state": (C.c_int, [P, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                             C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
            "lmfao_describe_plan": (C.c_int, [P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
            "lmfao_cart_variances": (C.c_int, [P, C.POINTER(C.c_int), C.c_int, P, P]),
            "lmfao_kernel_times": (C.c_int, [P, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]),
            "lmfao_kernel_name": (C.c_char_p, [P, C.c_int]),
            "lmfao_set_profiling": (C.c_int, [P, C.c_int]),
            "lmfao_cart_variances_noalloc": (C.c_int, [P, C.POINTER(C.c_int), C.c_int, P, P]),
            "lmfao_mlp_param_count": (C.c_int64, [C.c_int]),
            "lmfao_plan_candidates": (C.c_int, [P, C.POINTER(PlanOpts), C.POINTER(C.c_int32), C.POINTER(C.c_float),
                                                C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "lmfao_mlp_forward": (C.c_int, [P, C.c_int, C.c_int, P, P, P, P, P]),
            "lmfao_mlp_loss": (C.c_int, [P, P, C.c_int, P, P, P]),
            "lmfao_mlp_backward": (C.c_int, [P, C.c_int, C.c_int, P, P, P, P, P, P]),
            "lmfao_mlp_adam": (C.c_int, [P, P, P, P, C.c_int64, C.c_int, C.c_float, P]),
            "lmfao_group_count": (C.c_int, [P, C.POINTER(GroupBy), C.c_int, C.c_int64, P, P, C.POINTER(C.c_int64)]),
            "lmfao_ridge_fit": (C.c_int, [P, C.c_int, C.c_char_p, C.POINTER(C.c_char_p), C.c_int, C.c_double, C.c_int,
                                          C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]),
            "lmfao_cart_tree": (C.c_int, [P, C.c_char_p, C.POINTER(C.c_char_p), C.c_int, C.POINTER(C.c_float),
                                          C.POINTER(C.c_int32), C.c_int, C.POINTER(PlanOpts), C.POINTER(CartNode),
                                          C.POINTER(C.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class _DeviceArray:
    """A borrowed device array, exposed through the CUDA array interface."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _wrap_device(ptr, n, typestr, dtype, device):
    import torch
    if n == 0:
        return torch.zeros(0, dtype=dtype, device=device)
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device=device)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class Engine:
    """One engine context on a CUDA device (``lmfao_create``)."""

    def __init__(self, device=0):
        self.lib = library()
        self.ctx = C.c_void_p()
        rc = self.lib.lmfao_create(C.byref(self.ctx), int(device))
        if rc != OK:
            raise LmfaoError(rc, "lmfao_create failed (no usable CUDA device?)")
        self.device = int(device)
        self.rel_ids = {}
        self.queries = []
        self._keep = []

    # ------------------------------------------------------------------ plumbing
    def _check(self, rc):
        if rc != OK:
            raise LmfaoError(rc, self.lib.lmfao_last_error(self.ctx).decode())

    def close(self):
        if self.ctx:
            self.lib.lmfao_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ relations
    def load_relation(self, rel, where="host"):
        """Load a relation in the ``workloads`` vocabulary. Column data are numpy arrays
        (``where="host"``) or CUDA tensors (``"device"`` copies, ``"adopt"`` borrows)."""
        cols = (Column * len(rel["columns"]))()
        keep = []
        for i, c in enumerate(rel["columns"]):
            data = c["data"]
            role = ROLE[c["role"]]
            if where == "host":
                arr = np.ascontiguousarray(data)
                if role in (KEY, CAT):
                    arr = arr.astype(np.int32, copy=False)
                    dt = I32
                elif arr.dtype == np.uint8:
                    dt = U8
                else:
                    arr = arr.astype(np.float32, copy=False)
                    dt = F32
                keep.append(arr)
                ptr = arr.ctypes.data
            else:
                t = data
                dt = {"torch.int32": I32, "torch.float32": F32, "torch.uint8": U8}[str(t.dtype)]
                if not t.is_contiguous():
                    raise ValueError("device columns must be contiguous")
                keep.append(t)
                ptr = t.data_ptr()
            name = c["attr"].encode()
            keep.append(name)
            cols[i] = Column(name, dt, role, int(c.get("domain", 0)), C.c_void_p(ptr))
        rid = C.c_int()
        flags = {"host": HOST, "device": DEVICE, "adopt": ADOPT_DEVICE}[where]
        self._check(self.lib.lmfao_load_relation(self.ctx, rel["name"].encode(), int(rel["nrows"]), cols,
                                                 len(rel["columns"]), flags, C.byref(rid)))
        if where == "adopt":
            self._keep.append(keep)
        self.rel_ids[rel["name"]] = rid.value
        return rid.value

    # ------------------------------------------------------------------ batch
    def add_query(self, q):
        keep = []
        aggs = (Aggregate * max(1, len(q["aggs"])))()
        for i, agg in enumerate(q["aggs"]):
            fs = (Factor * max(1, len(agg)))()
            for j, (attr, fn, p) in enumerate(agg):
                b = attr.encode()
                keep.append(b)
                fs[j] = Factor(b, FN_POW if fn == "pow" else FN_ID, int(p))
            keep.append(fs)
            aggs[i] = Aggregate(fs, len(agg))
        gbs = (GroupBy * max(1, len(q.get("groupby", []))))()
        for i, (attr, kind, thr) in enumerate(q.get("groupby", [])):
            b = attr.encode()
            keep.append(b)
            if kind == "bucket":
                t = np.ascontiguousarray(thr, dtype=np.float32)
                keep.append(t)
                gbs[i] = GroupBy(b, GB_BUCKET, len(t), t.ctypes.data_as(C.POINTER(C.c_float)))
            else:
                gbs[i] = GroupBy(b, GB_VALUE, 0, None)
        prs = (Predicate * max(1, len(q.get("filters", []))))()
        for i, (attr, op, t) in enumerate(q.get("filters", [])):
            b = attr.encode()
            keep.append(b)
            prs[i] = Predicate(b, OPS[op], float(np.float32(t)))
        qid = C.c_int()
        self._check(self.lib.lmfao_add_batch(self.ctx, aggs, len(q["aggs"]), gbs, len(q.get("groupby", [])), prs,
                                             len(q.get("filters", [])), C.byref(qid)))
        self.queries.append(q)
        return qid.value

    def add_queries(self, qs):
        return [self.add_query(q) for q in qs]

    def clear_batch(self):
        self._check(self.lib.lmfao_clear_batch(self.ctx))
        self.queries = []

    # ------------------------------------------------------------------ plan / run / fetch
    def plan(self, precision="fp32", planner="heuristic", root=None, segment="default", mode="auto",
             join_parent=None, query_roots=None, autotune=False, cost_model=None, combine="auto", learned_topk=1):
        o = PlanOpts()
        o.learned_topk = int(learned_topk)
        o.precision = PRECISION[precision]
        forced = root is not None or segment != "default" or planner == "forced"
        o.planner = PLANNER["forced" if forced and planner == "heuristic" else planner]
        o.root_rel = -1 if root is None else (self.rel_ids[root] if isinstance(root, str) else int(root))
        if segment == "default":
            o.segment_rel = -2
        elif segment is None:
            o.segment_rel = -1
        else:
            o.segment_rel = self.rel_ids[segment] if isinstance(segment, str) else int(segment)
        o.mode = MODE[mode]
        o.autotune = 1 if autotune else 0
        o.combine = {"auto": 0, "entry": 1, "block": 2}[combine]
        keep = []
        if join_parent is not None:
            arr = (C.c_int32 * len(join_parent))(*[int(x) for x in join_parent])
            keep.append(arr)
            o.join_parent = arr
        if query_roots is not None:
            arr = (C.c_int32 * len(query_roots))(*[int(x) for x in query_roots])
            keep.append(arr)
            o.query_root = arr
        if cost_model is None and planner == "learned":
            cost_model = COST_MODEL_PATH
        if cost_model is not None:
            b = cost_model.encode()
            keep.append(b)
            o.cost_model = b
        info = PlanInfo()
        self._check(self.lib.lmfao_plan(self.ctx, C.byref(o), C.byref(info)))
        return {f: getattr(info, f) for f, _ in PlanInfo._fields_}

    def plan_candidates(self, precision="fp32", join_parent=None):
        """Candidate physical plans (n x 4: root, segment, mode, combine) and their features."""
        o = PlanOpts()
        o.precision = PRECISION[precision]
        o.planner = PLANNER["heuristic"]
        o.root_rel = -1
        o.segment_rel = -2
        keep = None
        if join_parent is not None:
            keep = (C.c_int32 * len(join_parent))(*[int(x) for x in join_parent])
            o.join_parent = keep
        n = C.c_int()
        nf = C.c_int()
        self._check(self.lib.lmfao_plan_candidates(self.ctx, C.byref(o), None, None, 0, C.byref(n), C.byref(nf)))
        cand = (C.c_int32 * (4 * max(1, n.value)))()
        feats = (C.c_float * (nf.value * max(1, n.value)))()
        self._check(self.lib.lmfao_plan_candidates(self.ctx, C.byref(o), cand, feats, n.value, C.byref(n),
                                                   C.byref(nf)))
        c = np.ctypeslib.as_array(cand)[:4 * n.value].reshape(n.value, 4).copy()
        f = np.ctypeslib.as_array(feats)[:nf.value * n.value].reshape(n.value, nf.value).copy()
        return c, f

    def plan_candidate(self, cand, precision="fp32", join_parent=None):
        root, seg, mode, comb = [int(v) for v in cand]
        return self.plan(precision=precision, planner="forced", root=root, segment=None if seg == -1 else seg,
                         mode={0: "auto", 1: "factorised", 2: "per_tuple", 3: "generic"}[mode],
                         combine={0: "auto", 1: "entry", 2: "block"}[comb], join_parent=join_parent)

    def run(self, stream=None):
        self._check(self.lib.lmfao_run(self.ctx, _stream_handle(stream)))

    def fetch(self, qid):
        """Result of a query in the oracle's format: keys (ngroups x ngroupby, int64),
        counts (int64), sums (ngroups x naggs, float64)."""
        r = Result()
        self._check(self.lib.lmfao_fetch(self.ctx, int(qid), C.byref(r)))
        ng, nb, na = r.ngroups, r.ngroupby, r.naggs
        keys = np.ctypeslib.as_array(r.group_keys, shape=(ng * nb,)).reshape(ng, nb).astype(np.int64) \
            if ng * nb else np.zeros((ng, nb), dtype=np.int64)
        counts = np.ctypeslib.as_array(r.counts, shape=(ng,)).copy() if ng else np.zeros(0, dtype=np.int64)
        sums = np.ctypeslib.as_array(r.sums, shape=(ng * na,)).reshape(ng, na).copy() if ng * na else \
            np.zeros((ng, na))
        return {"keys": keys, "counts": counts.astype(np.int64), "sums": sums}

    def fetch_all(self):
        return [self.fetch(i) for i in range(len(self.queries))]

    def result_cells(self, qid):
        n = C.c_int64()
        self._check(self.lib.lmfao_result_device(self.ctx, int(qid), None, None, C.byref(n), None))
        return n.value

    def result_device(self, qid, counts, sums, stream=None):
        """Dense device results into CUDA tensors (int64 counts, float64 sums)."""
        n = C.c_int64()
        self._check(self.lib.lmfao_result_device(
            self.ctx, int(qid), C.c_void_p(counts.data_ptr()) if counts is not None else None,
            C.c_void_p(sums.data_ptr()) if sums is not None else None, C.byref(n), _stream_handle(stream)))
        return n.value

    def result_state(self):
        """The plan's result arrays (int64 counts, float64 sums) as CUDA tensors that share the
        engine's memory: sum them over the shards of a data-parallel run before fetching."""
        import torch
        pc, ps = C.c_void_p(), C.c_void_p()
        nc, ns = C.c_int64(), C.c_int64()
        self._check(self.lib.lmfao_result_state(self.ctx, C.byref(pc), C.byref(nc), C.byref(ps), C.byref(ns)))
        dev = torch.device("cuda", self.device)
        return (_wrap_device(pc.value, nc.value, "<i8", torch.int64, dev),
                _wrap_device(ps.value, ns.value, "<f8", torch.float64, dev))

    def describe(self):
        need = C.c_size_t()
        self._check(self.lib.lmfao_describe_plan(self.ctx, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        self._check(self.lib.lmfao_describe_plan(self.ctx, buf, need.value, C.byref(need)))
        return json.loads(buf.value.decode())

    def cart_variances(self, qids, out, stream=None):
        arr = (C.c_int * len(qids))(*[int(q) for q in qids])
        self._check(self.lib.lmfao_cart_variances(self.ctx, arr, len(qids), C.c_void_p(out.data_ptr()),
                                                  _stream_handle(stream)))

    def group_count(self, groupby, cap):
        """COUNT GROUP BY ``groupby`` (list of (attr, "value"|"bucket", thresholds)) with hash-table
        results (lmfao_group_count). Returns (codes: n x ngb int64, counts: n int64, groups) with
        n = min(groups, cap); FP32 values come back as their 32-bit patterns (non-negative)."""
        import torch
        keep = []
        gbs = (GroupBy * len(groupby))()
        for i, (attr, kind, thr) in enumerate(groupby):
            b = attr.encode()
            keep.append(b)
            if kind == "bucket":
                t = np.ascontiguousarray(np.asarray(thr, dtype=np.float32))
                keep.append(t)
                gbs[i] = GroupBy(b, GB_BUCKET, len(t), t.ctypes.data_as(C.POINTER(C.c_float)))
            else:
                gbs[i] = GroupBy(b, GB_VALUE, 0, None)
        keys = torch.empty((max(1, cap), len(groupby)), dtype=torch.int32, device="cuda")
        counts = torch.empty(max(1, cap), dtype=torch.int64, device="cuda")
        n = C.c_int64()
        self._check(self.lib.lmfao_group_count(self.ctx, gbs, len(groupby), int(cap), C.c_void_p(keys.data_ptr()),
                                               C.c_void_p(counts.data_ptr()), C.byref(n)))
        m = min(n.value, cap)
        k = keys[:m].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
        return k, counts[:m].cpu().numpy(), n.value

    def ridge_fit(self, qid, target, features, lam, method="closed_form", iters=0, step=0.0):
        """Ridge regression from query ``qid``'s aggregates (lmfao_ridge_fit). Returns
        (theta with the intercept first, J(theta), |grad J(theta)|)."""
        names = (C.c_char_p * max(1, len(features)))(*[f.encode() for f in features])
        th = (C.c_double * (len(features) + 1))()
        loss, gn = C.c_double(), C.c_double()
        self._check(self.lib.lmfao_ridge_fit(self.ctx, int(qid), target.encode(), names, len(features), float(lam),
                                             {"closed_form": 0, "bgd": 1}[method], int(iters), float(step), th,
                                             C.byref(loss), C.byref(gn)))
        return np.array(th[:]), loss.value, gn.value

    def cart_tree(self, target, features, thresholds, depth, precision="fp32"):
        """Grow a regression tree (lmfao_cart_tree). ``thresholds``: dict or list of ascending
        thresholds per feature. Returns (nodes in heap order as dicts, per-level [plan_ms, run_ms])."""
        thr = [np.asarray(thresholds[f] if isinstance(thresholds, dict) else thresholds[i], dtype=np.float32)
               for i, f in enumerate(features)]
        names = (C.c_char_p * len(features))(*[f.encode() for f in features])
        flat = np.ascontiguousarray(np.concatenate(thr).astype(np.float32))
        counts = (C.c_int32 * len(features))(*[len(t) for t in thr])
        o = PlanOpts()
        o.precision = PRECISION[precision]
        o.planner = PLANNER["heuristic"]
        o.root_rel = -1
        o.segment_rel = -2
        nn = (1 << depth) - 1
        nodes = (CartNode * nn)()
        ms = (C.c_double * (2 * depth))()
        self._check(self.lib.lmfao_cart_tree(self.ctx, target.encode(), names, len(features),
                                             flat.ctypes.data_as(C.POINTER(C.c_float)), counts, depth, C.byref(o),
                                             nodes, ms))
        self.queries = []
        out = [{f: getattr(nodes[i], f) for f, _ in CartNode._fields_} for i in range(nn)]
        return out, [[ms[2 * i], ms[2 * i + 1]] for i in range(depth)]

    def cart_variances_noalloc(self, qids, out, stream=None):
        """Same as ``cart_variances`` without any device allocation (fixed descriptor
        array of LMFAO_NOALLOC_MAX_QUERIES entries shared by all calls on the device)."""
        arr = (C.c_int * max(1, len(qids)))(*[int(q) for q in qids])
        self._check(self.lib.lmfao_cart_variances_noalloc(self.ctx, arr, len(qids), C.c_void_p(out.data_ptr()),
                                                          _stream_handle(stream)))

    def set_profiling(self, on=True):
        self._check(self.lib.lmfao_set_profiling(self.ctx, 1 if on else 0))

    def kernel_times(self):
        ms = (C.c_double * 256)()
        n = C.c_int()
        self._check(self.lib.lmfao_kernel_times(self.ctx, ms, 256, C.byref(n)))
        return [(self.lib.lmfao_kernel_name(self.ctx, i).decode(), ms[i]) for i in range(n.value)]


class CostModel:
    """The planner's cost model: a 3-layer, 64-wide perceptron whose forward, backward and
    Adam kernels are in liblmfao.so. Tensors are torch CUDA float32 tensors."""

    def __init__(self, d, seed=0, device="cuda"):
        import torch
        self.lib = library()
        self.d = d
        n = self.lib.lmfao_mlp_param_count(d)
        if n < 0:
            raise LmfaoError(ERR_ARG, "feature count must be in [1, 256]")
        g = torch.Generator().manual_seed(seed)
        p = torch.zeros(n)
        h = 64
        w1 = torch.randn(d, h, generator=g) * (2.0 / d) ** 0.5
        w2 = torch.randn(h, h, generator=g) * (2.0 / h) ** 0.5
        w3 = torch.randn(h, generator=g) * (1.0 / h) ** 0.5
        o = 0
        p[o:o + d * h] = w1.reshape(-1); o += d * h
        o += h
        p[o:o + h * h] = w2.reshape(-1); o += h * h
        o += h
        p[o:o + h] = w3; o += h
        self.params = p.to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0

    def _ptr(self, t):
        return C.c_void_p(t.data_ptr()) if t is not None else None

    def forward(self, x, keep=False, stream=None):
        import torch
        n = x.shape[0]
        y = torch.empty(n, device=x.device)
        h1 = torch.empty(n, 64, device=x.device) if keep else None
        h2 = torch.empty(n, 64, device=x.device) if keep else None
        rc = self.lib.lmfao_mlp_forward(self._ptr(x), n, self.d, self._ptr(self.params), self._ptr(h1), self._ptr(h2),
                                        self._ptr(y), _stream_handle(stream))
        if rc != OK:
            raise LmfaoError(rc, "lmfao_mlp_forward")
        return (y, h1, h2) if keep else y

    def backward(self, x, h1, h2, gy, stream=None):
        rc = self.lib.lmfao_mlp_backward(self._ptr(x), x.shape[0], self.d, self._ptr(self.params), self._ptr(h1),
                                         self._ptr(h2), self._ptr(gy), self._ptr(self.grad), _stream_handle(stream))
        if rc != OK:
            raise LmfaoError(rc, "lmfao_mlp_backward")
        return self.grad

    def train_step(self, x, t, lr=1e-3, stream=None):
        import torch
        y, h1, h2 = self.forward(x, keep=True, stream=stream)
        gy = torch.empty_like(y)
        loss = torch.zeros(1, device=x.device)
        rc = self.lib.lmfao_mlp_loss(self._ptr(y), self._ptr(t), x.shape[0], self._ptr(gy), self._ptr(loss),
                                     _stream_handle(stream))
        if rc != OK:
            raise LmfaoError(rc, "lmfao_mlp_loss")
        self.backward(x, h1, h2, gy, stream)
        self.step += 1
        rc = self.lib.lmfao_mlp_adam(self._ptr(self.params), self._ptr(self.grad), self._ptr(self.m), self._ptr(self.v),
                                     self.params.numel(), self.step, float(lr), _stream_handle(stream))
        if rc != OK:
            raise LmfaoError(rc, "lmfao_mlp_adam")
        return loss


def load_workload(engine, rels, queries, where="host"):
    for R in rels:
        engine.load_relation(R, where)
    return engine.add_queries(queries)
