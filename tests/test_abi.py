"""The C-ABI library loads and exports every entry point declared in include/lmfao.h;
host-side argument checking works without a GPU (host-only context)."""
import os
import re

import numpy as np
import pytest

from paper_2008_08657_b300 import lmfao as L
from paper_2008_08657_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    txt = open(os.path.join(ROOT, "include", "lmfao.h")).read()
    return sorted(set(re.findall(r"LMFAO_API\s+(?:const\s+char\s*\*|int64_t|int)\s*(lmfao_\w+)\s*\(", txt)))


def test_library_exports_every_declared_entry_point():
    lib = L.library()
    names = declared_entry_points()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.ENTRY_POINTS) == names


def test_host_only_context_validates_arguments():
    e = L.Engine(device=-1)
    rels = W.star_schema(n_fact=100)
    for R in rels:
        e.load_relation(R)
    with pytest.raises(L.LmfaoError) as ei:
        e.add_query({"aggs": [[("nope", "id", 1)]], "groupby": [], "filters": []})
    assert ei.value.code == L.ERR_ARG
    with pytest.raises(L.LmfaoError) as ei:
        e.add_query({"aggs": [[]], "groupby": [("y", "value", None)], "filters": []})
    assert ei.value.code == L.ERR_ARG
    bad = W.relation("B", [W.column("a", np.array([0, 5000], dtype=np.int32), "key", 1000)])
    with pytest.raises(L.LmfaoError) as ei:
        e.load_relation(bad)
    assert ei.value.code == L.ERR_KEY_RANGE
    e.add_query({"aggs": [[]], "groupby": [], "filters": []})
    with pytest.raises(L.LmfaoError) as ei:
        e.run()
    assert ei.value.code == L.ERR_NOT_PLANNED
    e.close()


def test_dtype_rules():
    e = L.Engine(device=-1)
    R = W.relation("R", [W.column("a", np.zeros(3, dtype=np.float32), "key", 4)])
    cols = (L.Column * 1)()
    data = np.zeros(3, dtype=np.float32)
    cols[0] = L.Column(b"a", L.F32, L.KEY, 4, data.ctypes.data)
    rid = L.C.c_int()
    rc = e.lib.lmfao_load_relation(e.ctx, b"R", 3, cols, 1, L.HOST, L.C.byref(rid))
    assert rc == L.ERR_DTYPE
    e.close()
    assert R["nrows"] == 3


def test_create_on_missing_device_fails_cleanly():
    lib = L.library()
    ctx = L.C.c_void_p()
    rc = lib.lmfao_create(L.C.byref(ctx), 4096)
    assert rc == L.ERR_CUDA and not ctx.value


def test_options_without_an_implementation_are_refused():
    """A precision or tuning request this build cannot honour is refused with
    ERR_UNSUPPORTED (never silently replaced by another mode); unknown values are ERR_ARG."""
    e = L.Engine(device=-1)
    for R in W.star_schema(n_fact=100):
        e.load_relation(R)
    e.add_query({"aggs": [[]], "groupby": [], "filters": []})
    e.plan(precision="fp32")
    lib = L.library()
    o = L.PlanOpts()
    o.precision, o.planner, o.root_rel, o.segment_rel = 7, 0, -1, -2
    info = L.PlanInfo()
    assert lib.lmfao_plan(e.ctx, L.C.byref(o), L.C.byref(info)) == L.ERR_ARG
    o.precision, o.planner = 1, 9
    assert lib.lmfao_plan(e.ctx, L.C.byref(o), L.C.byref(info)) == L.ERR_ARG
    e.close()
