"""Engine against the oracle on the same seeded inputs (CUDA path through the C ABI)."""
import numpy as np
import pytest

from oracle import lmfao_oracle as O
from paper_2008_08657_b300 import workloads as W
from paper_2008_08657_b300.lmfao import ERR_ARG, ERR_UNSUPPORTED, Engine, LmfaoError
from tests.parity import compare

pytestmark = pytest.mark.gpu

# group-by attributes determined by the join key of their relation toward the root R0
# (R1 has distinct k1 values; R3's g3 would pass through R2, whose k2 values repeat)
TINY_GROUPS = ["k1", "k2", "g0", "g1"]
TINY_BUCKETS = ["x0", "x1"]


def run_engine(rels, qs, **plan):
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_queries(qs)
    info = e.plan(**plan)
    e.run()
    out = e.fetch_all()
    e.close()
    return out, info


# (seed, forced segment relation): R4 exists only in the five-relation variant (odd seeds)
TINY_SEG_CASES = [(seed, seg) for seed in range(16) for seg in (None, "R1", "R2", "R4")
                  if seg != "R4" or seed % 2 == 1]


@pytest.mark.parametrize("seed,segment", TINY_SEG_CASES)
@pytest.mark.parametrize("precision", ["fp32", "fp64", "split_bf16"])
@pytest.mark.parametrize("mode", ["factorised", "generic", "per_tuple"])
def test_tiny_schemas_match_oracle(seed, precision, mode, segment):
    shared3 = seed % 2 == 1
    rels = W.tiny_schema(seed, shared3=shared3, fd=True)
    qs = W.tiny_queries(seed, rels, nq=6, group_attrs=TINY_GROUPS, bucket_attrs=TINY_BUCKETS)
    ref = O.evaluate(rels, qs)
    # join tree: R1, R2, R4 below R0 and R3 below R2; the segment relation is forced
    parent = [-1, 0, 0, 2, 0][:len(rels)]
    got, _ = run_engine(rels, qs, precision=precision, mode=mode, root="R0", segment=segment,
                        join_parent=parent)
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"seed {seed} query {i}")


@pytest.mark.parametrize("lanes", ["0", "1"])
@pytest.mark.parametrize("seed,segment", [(a, b) for a, b in TINY_SEG_CASES if b is not None])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tiny_schemas_generated_root_pass(seed, precision, segment, lanes, monkeypatch):
    """Tiny schemas (duplicate and dangling keys, group-bys, buckets, filters) with the root
    pass generated at plan time at any size, in both lane layouts (segments far shorter than
    a warp's step); shapes outside the generator keep the template."""
    monkeypatch.setenv("LMFAO_CODEGEN", "1")
    monkeypatch.setenv("LMFAO_ROOT_LANES", lanes)
    shared3 = seed % 2 == 1
    rels = W.tiny_schema(seed, shared3=shared3, fd=True)
    qs = W.tiny_queries(seed, rels, nq=6, group_attrs=TINY_GROUPS, bucket_attrs=TINY_BUCKETS)
    ref = O.evaluate(rels, qs)
    parent = [-1, 0, 0, 2, 0][:len(rels)]
    got, _ = run_engine(rels, qs, precision=precision, mode="factorised", root="R0", segment=segment,
                        join_parent=parent)
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"seed {seed} query {i}")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_star_config_full_size(precision):
    rels = W.star_schema()
    qs = W.star_batch()
    ref = O.evaluate(rels, qs)
    got, info = run_engine(rels, qs, precision=precision)
    assert info["segment_rel"] >= 0
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"query {i}")
    assert got[0]["counts"][0] == 200_000


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("combine", ["block", "entry"])
def test_retailer_scaled(precision, combine):
    rels = W.retailer_schema(n_fact=1_000_000)
    qs = W.retailer_batch()
    ref = O.evaluate(rels, qs)
    got, info = run_engine(rels, qs, precision=precision, combine=combine)
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"query {i}")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_favorita_scaled_fig2_tree(precision):
    rels = W.favorita_schema(n_fact=300_000)
    qs = W.favorita_batch()
    names = [R["name"] for R in rels]
    parent = [names.index(W.FAVORITA_TREE[n]) if n in W.FAVORITA_TREE else -1 for n in names]
    ref = O.evaluate(rels, qs)
    got, info = run_engine(rels, qs, precision=precision, join_parent=parent)
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"query {i}")


@pytest.mark.parametrize("which", ["star", "retailer", "favorita"])
def test_benchmark_shapes_use_the_lean_root_pass(which):
    rels = {"star": lambda: W.star_schema(n_fact=50_000), "retailer": lambda: W.retailer_schema(n_fact=1_000_000),
            "favorita": lambda: W.favorita_schema(n_fact=2_000_000)}[which]()
    qs = {"star": W.star_batch, "retailer": W.retailer_batch, "favorita": W.favorita_batch}[which]()
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_queries(qs)
    e.plan()
    phys = e.describe()["physical"]
    e.close()
    assert phys["specialised_pass"] and phys["lean_pass"] and phys["per_tuple_items"] == 0
    if which == "retailer":
        assert phys["block_combine"] and phys["prefix_digits"] == 1


def test_plan_invariance_retailer():
    rels = W.retailer_schema(n_fact=200_000)
    qs = W.retailer_batch()[:4]
    base, _ = run_engine(rels, qs, precision="fp32")
    for plan in ({"segment": None}, {"segment": "Location"}, {"mode": "per_tuple"}, {"mode": "generic"},
                 {"precision": "fp64"}, {"combine": "entry"}):
        kw = {"precision": "fp32", **plan}
        other, _ = run_engine(rels, qs, **kw)
        for q, a, b in zip(qs, base, other):
            np.testing.assert_array_equal(a["keys"], b["keys"])
            np.testing.assert_array_equal(a["counts"], b["counts"])
            scale = np.maximum(np.abs(a["sums"]), 1.0)
            assert (np.abs(a["sums"] - b["sums"]) <= 1e-4 * scale).all(), plan


@pytest.mark.parametrize("n_fact,mode,codegen", [(300_000, "auto", "0"), (1_000_000, "auto", "0"),
                                                 (1_000_000, "auto", "1"), (1_000_000, "generic", "0")])
def test_dt_level_and_cart_variances(n_fact, mode, codegen, monkeypatch):
    """A decision-tree level (8 leaves as a filter family); codegen "1" runs the root pass
    generated at plan time, "0" the template kernel."""
    import torch
    monkeypatch.setenv("LMFAO_CODEGEN", codegen)
    rels = W.retailer_schema(n_fact=n_fact)
    qs, splits, thr = W.dt_level_batch(rels)
    ref = O.evaluate(rels, qs)
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_queries(qs)
    e.plan(precision="fp32", mode=mode)
    phys = e.describe()["physical"]
    if n_fact >= 1_000_000 and mode == "auto":
        assert phys["filter_family"] == 8 and phys["per_tuple_items"] == 0
        assert phys["root_pass"]["generated"] == (codegen == "1"), phys["root_pass"]["not_generated_because"]
    e.run()
    got = e.fetch_all()
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"query {i}")
    nb = max(len(t) for t in thr.values()) + 1
    ids = [i for i, q in enumerate(qs) if len(q["groupby"][0][2]) + 1 == nb]
    out = torch.zeros((len(ids), nb - 1, 2), dtype=torch.float64, device="cuda")
    e.cart_variances(ids, out)
    torch.cuda.synchronize()
    for k, qi in enumerate(ids):
        left, right = O.cart_variances(ref[qi])
        nbq = len(left)
        L = out[k, :nbq, 0].cpu().numpy()
        R_ = out[k, :nbq, 1].cpu().numpy()
        scale = np.abs(ref[qi]["abs"][:, 2]).sum() + 1.0
        assert np.abs(L - left).max() <= 1e-5 * scale
        assert np.abs(R_ - right).max() <= 1e-5 * scale
    e.close()


def test_cart_variances_check_and_map_their_aggregates():
    """lmfao_cart_variances needs COUNT, SUM(y), SUM(y^2) of one attribute: the three in any
    order give the same variances; other aggregates are refused with ERR_ARG."""
    import torch
    rels = W.retailer_schema(n_fact=50_000, seed=2)
    ycol, x = "y", "i1"
    item = next(R for R in rels if R["name"] == "Item")
    xthr = [float(v) for v in np.quantile(next(c["data"] for c in item["columns"] if c["attr"] == x),
                                          [0.25, 0.5, 0.75])]
    gb = [(x, "bucket", xthr)]
    canon = {"aggs": [[], [(ycol, "id", 1)], [(ycol, "pow", 2)]], "groupby": gb, "filters": []}
    perm = {"aggs": [[(ycol, "id", 1), (ycol, "id", 1)], [], [(ycol, "id", 1)]], "groupby": gb, "filters": []}
    other = {"aggs": [[], [(x, "id", 1)], [(ycol, "pow", 2)]], "groupby": gb, "filters": []}
    four = {"aggs": [[], [(ycol, "id", 1)], [(ycol, "pow", 2)], []], "groupby": gb, "filters": []}
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_queries([canon, perm, other, four])
    e.plan(precision="fp32")
    e.run()
    ref = O.evaluate(rels, [canon])[0]
    left, right = O.cart_variances(ref)
    out = torch.zeros((2, len(xthr), 2), dtype=torch.float64, device="cuda")
    e.cart_variances([0, 1], out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    scale = np.abs(ref["abs"][:, 2]).sum() + 1.0
    for k in range(2):
        assert np.abs(got[k, :len(left), 0] - left).max() <= 1e-5 * scale
        assert np.abs(got[k, :len(right), 1] - right).max() <= 1e-5 * scale
    for bad in (2, 3):
        for call in (e.cart_variances, e.cart_variances_noalloc):
            with pytest.raises(LmfaoError) as ei:
                call([0, bad], out)
            assert ei.value.code == ERR_ARG
    e.close()


def test_group_attribute_not_determined_by_key_is_reported():
    rels = W.tiny_schema(3, empty_ok=False)  # R1 keys repeat, so g1 is not a function of k1
    rels[1]["columns"][0]["data"][:] = 0
    rels[1]["columns"][2]["data"][:] = np.arange(rels[1]["nrows"]) % 2
    q = {"aggs": [[]], "groupby": [("g1", "value", None)], "filters": []}
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_query(q)
    with pytest.raises(LmfaoError) as ei:  # detected on the loaded data when the plan is built
        e.plan(root="R0")
    assert ei.value.code == ERR_UNSUPPORTED and "not determined" in str(ei.value)
    e.close()


def test_heuristic_planner_avoids_a_root_that_leaves_a_group_by_undetermined():
    """With 50k fact tuples the largest relation is Weather; rooted there, Item's bucketed
    attribute would reach the root through Inventory's view keyed by (locn, date), which does
    not determine it. The heuristic planner moves the root and the results equal the oracle;
    forcing the Weather root is refused when planning."""
    rels = W.retailer_schema(n_fact=50_000, seed=2)
    item = next(R for R in rels if R["name"] == "Item")
    thr = [float(v) for v in np.quantile(next(c["data"] for c in item["columns"] if c["attr"] == "i1"),
                                         [0.25, 0.5, 0.75])]
    qs = [{"aggs": [[], [("y", "id", 1)], [("y", "pow", 2)]], "groupby": [("i1", "bucket", thr)], "filters": []}]
    ref = O.evaluate(rels, qs)
    e = Engine(0)
    for R in rels:
        e.load_relation(R)
    e.add_queries(qs)
    with pytest.raises(LmfaoError) as ei:
        e.plan(root="Weather")
    assert ei.value.code == ERR_UNSUPPORTED
    e.plan()
    assert e.describe()["physical"]["root"] != "Weather"
    e.run()
    compare(qs[0], e.fetch(0), ref[0])
    e.close()


def test_empty_fact_and_empty_dimension():
    rels = W.star_schema(n_fact=0)
    qs = W.star_batch()
    got, _ = run_engine(rels, qs)
    ref = O.evaluate(rels, qs)
    for q, g, r in zip(qs, got, ref):
        compare(q, g, r)
    rels = W.star_schema(n_fact=1000)
    rels[2] = W.relation("D2", [dict(c, data=c["data"][:0]) for c in rels[2]["columns"]])
    got, _ = run_engine(rels, qs)
    ref = O.evaluate(rels, qs)
    for q, g, r in zip(qs, got, ref):
        compare(q, g, r)
    assert got[0]["counts"][0] == 0


def test_device_columns_and_torch_stream():
    import torch
    rels = W.star_schema(n_fact=50_000)
    qs = W.star_batch()
    ref = O.evaluate(rels, qs)
    e = Engine(0)
    for R in rels:
        dev = dict(R, columns=[dict(c, data=torch.from_numpy(c["data"]).cuda()) for c in R["columns"]])
        e.load_relation(dev, where="adopt" if R["name"] == "F" else "device")
    e.add_queries(qs)
    e.plan()
    s = torch.cuda.Stream()
    e.run(s)
    got = e.fetch_all()
    for q, g, r in zip(qs, got, ref):
        compare(q, g, r)
    e.close()


@pytest.mark.parametrize("world", [2, 3])
def test_summed_shard_states_equal_the_whole_relation(world):
    """The data-parallel merge with the engine's own result state: one context per row shard
    of the fact relation (run one after another on this GPU), states summed element-wise
    into shard 0's, whose fetch then equals the oracle over the whole relation."""
    import torch
    from paper_2008_08657_b300.distributed import shard_relation
    rels = W.retailer_schema(n_fact=200_000, seed=4)
    qs = W.retailer_batch()
    ref = O.evaluate(rels, qs)
    engines = []
    try:
        for r in range(world):
            e = Engine(0)
            for R in rels:
                e.load_relation(shard_relation(R, r, world) if R is rels[0] else R)
            e.add_queries(qs)
            e.plan(root=rels[0]["name"])  # a shard may be smaller than Weather: keep the fact root
            e.run()
            engines.append(e)
        torch.cuda.synchronize()
        c0, s0 = engines[0].result_state()
        for e in engines[1:]:
            c, s = e.result_state()
            assert c.shape == c0.shape and s.shape == s0.shape
            c0 += c
            s0 += s
        torch.cuda.synchronize()
        got = engines[0].fetch_all()
    finally:
        for e in engines:
            e.close()
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"merged query {i}")


_SHAPES = {}


def _shape_case(which):
    """Benchmark-shaped inputs with ragged segments and their oracle results (computed once)."""
    if which not in _SHAPES:
        rels = {"star": lambda: W.star_schema(n_fact=60_001, seed=7),
                "retailer": lambda: W.retailer_schema(n_fact=1_000_003, seed=7),
                "favorita": lambda: W.favorita_schema(n_fact=2_000_003, seed=7)}[which]()
        qs = {"star": W.star_batch, "retailer": W.retailer_batch, "favorita": W.favorita_batch}[which]()
        _SHAPES[which] = (rels, qs, O.evaluate(rels, qs))
    return _SHAPES[which]


@pytest.mark.parametrize("codegen", ["0", "1", "lanes"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("which", ["star", "retailer", "favorita"])
def test_generated_and_template_root_pass_match_the_oracle(which, precision, codegen, monkeypatch):
    """The plan-specialised root pass (compiled at plan time) and the template kernel, on the
    benchmark shapes with ragged segments (head and tail tuples outside full quads); "lanes" is
    the generated pass in its one-tuple-per-lane layout (items of any length end inside the
    unrolled ring of loads)."""
    monkeypatch.setenv("LMFAO_CODEGEN", "0" if codegen == "0" else "1")
    monkeypatch.setenv("LMFAO_ROOT_LANES", "1" if codegen == "lanes" else "0")
    rels, qs, ref = _shape_case(which)
    e = Engine(0)
    try:
        for R in rels:
            e.load_relation(R)
        e.add_queries(qs)
        e.plan(precision=precision)
        phys = e.describe()["physical"]
        assert "root_pass" in phys and phys["lean_pass"], phys
        rp = phys["root_pass"]
        lanes = phys["tiles"]["root_pass_lanes"]
        e.run()
        got = e.fetch_all()
    finally:
        e.close()
    if codegen == "0":
        assert not rp["generated"]
    else:  # generated unless its table and partials exceed shared memory (FP64 Retailer)
        assert rp["generated"] or rp["not_generated_because"] == "shared memory", rp["not_generated_because"]
        assert rp["generated"] or precision == "fp64"
        if rp["generated"]:
            assert lanes == ("tuple per lane" if codegen == "lanes" else "quad per lane"), lanes
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"{which} {precision} codegen={codegen} query {i}")


_FAV = {}


@pytest.mark.parametrize("projection", ["stream", "kernels", False])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_favorita_projection_and_entry_combine(precision, projection, monkeypatch):
    """Favorita with the (date, store) segment key: outer store groups change inside every
    date block, so the combine is the projection combine (per-date and per-store projections
    of the per-segment sums, per-segment store x holiday cells; "stream": one pass over the
    sums in tiles with the per-segment entries fused, "kernels": one kernel per projection)
    or, with it switched off, the entry combine. The batch adds the Section 2 queries Q1-Q3
    (Q2 has a factor on the date key digit)."""
    if projection is False:
        monkeypatch.setenv("LMFAO_NO_PROJECTION_COMBINE", "1")
    else:
        monkeypatch.setenv("LMFAO_PROJECTION", projection)
    if not _FAV:
        rels = W.favorita_schema(n_fact=700_001, seed=3)
        qs = W.favorita_batch() + W.favorita_example_queries()
        _FAV["case"] = (rels, qs, O.evaluate(rels, qs))
    rels, qs, ref = _FAV["case"]
    e = Engine(0)
    try:
        for R in rels:
            e.load_relation(R)
        e.add_queries(qs)
        e.plan(precision=precision)
        phys = e.describe()["physical"]
        e.run()
        got = e.fetch_all()
    finally:
        e.close()
    assert phys["segment_relation"] == "Transactions" and not phys["block_combine"], phys
    assert phys["projection_combine"] == (projection is not False)
    assert phys["projection_stream"] == (projection == "stream"), phys
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"{precision} projection={projection} query {i}")


@pytest.mark.parametrize("precision,impl,chunk", [("fp32", "two", None), ("fp64", "two", None), ("fp32", "two", 16),
                                                  ("fp64", "two", 16), ("fp32", "dense", None), ("fp32", "dense", 16),
                                                  ("split_bf16", "two", None), ("fp32", "general", None),
                                                  ("fp64", "general", None), ("fp32", "single", None),
                                                  ("fp64", "single", None)])
def test_block_combine_kernels_match_the_oracle(precision, impl, chunk, monkeypatch):
    """The block combine as two kernels (per-block contraction into scratch, then the entries;
    FP32 and FP64 on the CUDA cores with the B operand read from the view rows: pipelined with
    cp.async ("two", the default) or with plain loads ("dense"), or built term by term
    ("general", TMA-staged sums); split BF16 on the tensor cores) and as the single-kernel form,
    on the Retailer shape with ragged segments: blocks of 124 segments run as chunks of 64 and
    60 (the last padded to the MMA's K), or of 16 (7 full, 12 left; the pipeline crosses block
    boundaries)."""
    monkeypatch.setenv("LMFAO_COMBINE", impl)
    if chunk:
        monkeypatch.setenv("LMFAO_COMBINE_CHUNK", str(chunk))
    rels, qs, ref = _shape_case("retailer")
    e = Engine(0)
    try:
        for R in rels:
            e.load_relation(R)
        e.add_queries(qs)
        e.plan(precision=precision)
        phys = e.describe()["physical"]
        # in FP64 the single-kernel block tables exceed shared memory: the entry combine runs
        assert phys["block_combine"] == (impl != "single" or precision != "fp64"), phys
        assert phys["block_combine_two_kernels"] == (impl != "single"), phys["combine_note"]
        if impl != "single":
            dense = impl in ("two", "dense") and precision != "split_bf16"
            assert phys["combine_bulk_copies"] == (not dense), phys
            want = {"fp32": "cuda cores FP32", "fp64": "cuda cores FP64",
                    "split_bf16": "tensor cores (tcgen05, split BF16)"}[precision]
            if dense:
                want += ", dense B operand" + (", cp.async pipeline" if impl == "two" else "")
            assert phys["contraction"] == want, phys
            assert phys["combine_chunk"] == (chunk or 64), phys
        e.run()
        got = e.fetch_all()
    finally:
        e.close()
    for i, (q, g, r) in enumerate(zip(qs, got, ref)):
        compare(q, g, r, where=f"query {i}")


@pytest.mark.parametrize("which", ["retailer", "dt"])
def test_autotuned_plans_match_the_oracle_and_reuse_their_tiles(which, tmp_path, monkeypatch):
    """Autotuning times a few work-item lengths and combine chunks on the data while planning;
    the tuned plan gives the oracle's results, and a second plan of the same shape takes its
    tiles from the cache file without timing."""
    monkeypatch.setenv("LMFAO_TUNE_CACHE", str(tmp_path / "tiles.txt"))
    monkeypatch.setenv("LMFAO_CODEGEN", "1")
    if which == "retailer":
        rels, qs, ref = _shape_case("retailer")
    else:
        rels = W.retailer_schema(n_fact=300_000, seed=8)
        qs = W.dt_level_batch(rels, seed=8)[0]
        ref = O.evaluate(rels, qs)
    for attempt in range(2):
        e = Engine(0)
        try:
            for R in rels:
                e.load_relation(R)
            e.add_queries(qs)
            e.plan(autotune=True)
            tiles = e.describe()["physical"]["tiles"]
            e.run()
            got = e.fetch_all()
        finally:
            e.close()
        assert tiles["autotuned"] and tiles["from_cache"] == (attempt == 1), tiles
        if attempt == 0:
            assert tiles["candidates"] >= 5, tiles
        for i, (q, g, r) in enumerate(zip(qs, got, ref)):
            compare(q, g, r, where=f"attempt {attempt} query {i}")


def test_queries_that_need_different_roots_get_one_plan_per_root():
    """F(a, b, x) with A(a, ga) and B(b, gb) whose join keys repeat with different ga / gb values:
    a group-by on ga is determined only when A is the root, one on gb only when B is, so no
    single root serves the batch. Each query takes its own root (Section 2: per-query roots),
    the engine runs one physical plan per root, and every result equals the oracle's."""
    r = np.random.default_rng(12)
    n = 5000
    F = W.relation("F", [W.column("a", r.integers(0, 40, n).astype(np.int32), "key", 40),
                         W.column("b", r.integers(0, 30, n).astype(np.int32), "key", 30),
                         W.column("x", r.standard_normal(n).astype(np.float32), "cont")])
    A = W.relation("A", [W.column("a", np.repeat(np.arange(40), 3).astype(np.int32), "key", 40),
                         W.column("ga", r.integers(0, 5, 120).astype(np.int32), "cat", 5),
                         W.column("xa", r.standard_normal(120).astype(np.float32), "cont")])
    B = W.relation("B", [W.column("b", np.repeat(np.arange(30), 2).astype(np.int32), "key", 30),
                         W.column("gb", r.integers(0, 4, 60).astype(np.int32), "cat", 4)])
    rels = [F, A, B]
    qs = [{"aggs": [[], [("x", "id", 1)], [("xa", "id", 1)]], "groupby": [("ga", "value", None)], "filters": []},
          {"aggs": [[], [("x", "pow", 2)]], "groupby": [("gb", "value", None)], "filters": []},
          {"aggs": [[], [("x", "id", 1), ("xa", "id", 1)]], "groupby": [], "filters": []}]
    ref = O.evaluate(rels, qs)
    e = Engine(0)
    try:
        for R in rels:
            e.load_relation(R)
        e.add_queries(qs)
        info = e.plan()
        desc = e.describe()
        e.run()
        got = e.fetch_all()
        with pytest.raises(LmfaoError) as ei:
            e.result_state()
        assert ei.value.code == ERR_UNSUPPORTED
    finally:
        e.close()
    assert info["n_roots"] >= 2, desc["physical_roots"]
    roots = {tuple(x["queries"]) if isinstance(x["queries"], list) else x["queries"]: x["root"]
             for x in desc["physical_roots"]}
    assert any(v == "A" for v in roots.values()) and any(v == "B" for v in roots.values()), roots
    assert desc["query_roots"][0] == "A" and desc["query_roots"][1] == "B"
    for i, (q, g, r_) in enumerate(zip(qs, got, ref)):
        compare(q, g, r_, where=f"query {i}")
