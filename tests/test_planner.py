"""View generation and grouping (Section 2, Fig. 2) on a host-only context.

The paper's running example: the Favorita schema with the join tree of Fig. 2, queries
Q1 = SUM(units), Q2 = SUM(g(item) * h(date)) GROUP BY store and Q3 = SUM(units * price)
GROUP BY class, with Sales as root of Q1 and Q2 and Items as root of Q3. After merging,
the plan has the directional views V_T->S, V_R->T, V_O->T, V_H->S, V_I->S and V_S->I,
partitioned with the queries into 7 groups whose dependency graph is Fig. 2 (right):
Group 6 = {Q1, Q2, V_S->I} at Sales, Group 7 = {Q3} at Items.
"""
import numpy as np
import pytest

from paper_2008_08657_b300 import lmfao as L
from paper_2008_08657_b300 import workloads as W

SHORT = {"Sales": "S", "Transactions": "T", "StoRes": "R", "Oil": "O", "Holidays": "H", "Items": "I"}


def favorita_engine():
    e = L.Engine(device=-1)
    rels = W.favorita_schema(n_fact=100_000)
    for R in rels:
        e.load_relation(R)
    e.add_queries(W.favorita_example_queries())
    names = [R["name"] for R in rels]
    parent = [names.index(W.FAVORITA_TREE[n]) if n in W.FAVORITA_TREE else -1 for n in names]
    return e, names, parent


def views_of(d):
    return {f"V_{SHORT[v['from']]}->{SHORT[v['to']]}" for v in d["views"]}


def test_fig2_views_and_groups_with_paper_roots():
    e, names, parent = favorita_engine()
    info = e.plan(join_parent=parent, query_roots=[names.index("Sales"), names.index("Sales"), names.index("Items")])
    d = e.describe()
    assert views_of(d) == {"V_T->S", "V_R->T", "V_O->T", "V_H->S", "V_I->S", "V_S->I"}
    assert info["n_views"] == 6 and info["n_groups"] == 7
    groups = d["groups"]
    vname = [f"V_{SHORT[v['from']]}->{SHORT[v['to']]}" for v in d["views"]]
    desc = [(SHORT[g["node"]], sorted(vname[v] for v in g["views"]), sorted(g["queries"])) for g in groups]
    # Groups 1-4: the leaf views; Group 5: V_T->S; Group 6 at Sales; Group 7 = Q3 at Items
    assert desc[:4] == [("R", ["V_R->T"], []), ("O", ["V_O->T"], []), ("H", ["V_H->S"], []), ("I", ["V_I->S"], [])]
    assert desc[4] == ("T", ["V_T->S"], [])
    assert desc[5] == ("S", ["V_S->I"], [0, 1])
    assert desc[6] == ("I", [], [2])
    # dependency graph of Fig. 2 (right)
    assert set(groups[4]["deps"]) == {0, 1}
    assert set(groups[5]["deps"]) == {2, 3, 4}
    assert set(groups[6]["deps"]) == {5}
    # one view per edge serves all three queries where the paper says so
    vts = [v for v in d["views"] if SHORT[v["from"]] == "T"][0]
    assert set(vts["queries"]) == {0, 1, 2}
    assert vts["key"] == ["date", "store"]
    e.close()


def test_heuristic_roots_follow_group_by_attribute():
    e, names, parent = favorita_engine()
    e.plan(join_parent=parent)
    d = e.describe()
    assert [SHORT[r] for r in d["query_roots"]] == ["S", "S", "I"]
    e.close()


def test_gyo_join_tree_and_cycle_detection():
    e = L.Engine(device=-1)
    for R in W.retailer_schema(n_fact=200_000):
        e.load_relation(R)
    e.add_queries(W.retailer_batch()[:1])
    e.plan()
    d = e.describe()
    assert d["join_tree"]["root"] == "Inventory"
    assert d["join_tree"]["parent"] == {"Item": "Inventory", "Location": "Inventory", "Census": "Location",
                                        "Weather": "Inventory"}
    e.close()
    # triangle R(a,b), S(b,c), T(c,a) has no join tree
    e = L.Engine(device=-1)
    z = np.zeros(2, dtype=np.int32)
    for name, attrs in (("R", "ab"), ("S", "bc"), ("T", "ca")):
        e.load_relation(W.relation(name, [W.column(a, z, "key", 2) for a in attrs]))
    e.add_query({"aggs": [[]], "groupby": [], "filters": []})
    with pytest.raises(L.LmfaoError) as ei:
        e.plan()
    assert ei.value.code == L.ERR_CYCLIC
    e.close()


def test_running_intersection_is_enforced_on_forced_trees():
    e = L.Engine(device=-1)
    rels = W.retailer_schema(n_fact=200_000)
    for R in rels:
        e.load_relation(R)
    e.add_queries(W.retailer_batch()[:1])
    names = [R["name"] for R in rels]
    # Census below Item breaks the zip path Location-Census
    parent = [-1, 0, 0, names.index("Item"), 0]
    with pytest.raises(L.LmfaoError) as ei:
        e.plan(join_parent=parent)
    assert ei.value.code == L.ERR_ARG
    e.close()
