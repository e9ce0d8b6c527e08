"""GHD planning (Sections 2.3, 3.2) and the SQL translation rules (Section
3.1) on the host: fractional covers, the chosen decompositions, the
tie-break order, selection pushdown, and the hypergraph of the six-relation
BI query.  No GPU."""
import pytest

from paper_1708_07859_b300 import ghd, sql

E = ghd.Edge


def test_fractional_edge_cover_numbers():
    tri = [(0, 1), (1, 2), (0, 2)]
    assert ghd.rho_star({0, 1, 2}, tri) == pytest.approx(1.5)
    assert ghd.rho_star({0, 1}, tri) == pytest.approx(1.0)
    cyc4 = [(0, 1), (1, 2), (2, 3), (0, 3)]
    assert ghd.rho_star({0, 1, 2, 3}, cyc4) == pytest.approx(2.0)
    assert ghd.rho_star({0, 1, 2, 3}, [(0, 1, 2, 3)]) == pytest.approx(1.0)


def q5_hypergraph():
    # o=0 c=1 n=2 s=3 r=4
    return ghd.Hypergraph(5, [E("F", (0, 3), 60_000_000), E("O", (0, 1), 15_000_000, True),
                              E("C", (1, 2), 1_500_000), E("S", (3, 2), 100_000), E("N", (2, 4), 25),
                              E("R", (4,), 5, True)], outputs=(2,))


def test_bi_query_gets_the_two_node_ghd_and_pushdowns():
    hg = q5_hypergraph()
    g = ghd.choose_ghd(hg)
    assert g.fhw == pytest.approx(2.0)
    root = g.root
    assert root.bag == frozenset({0, 1, 2, 3})
    assert sorted(hg.edges[i].name for i in root.edges) == ["C", "F", "S"]
    kids = {frozenset(c.bag): c for c in root.children}
    assert set(kids) == {frozenset({2, 4}), frozenset({0, 1})}
    assert kids[frozenset({0, 1})].selection_node and [hg.edges[i].name for i in kids[frozenset({0, 1})].edges] == ["O"]
    nr = kids[frozenset({2, 4})]
    assert [hg.edges[i].name for i in nr.edges] == ["N"]
    assert len(nr.children) == 1 and nr.children[0].selection_node and nr.children[0].bag == frozenset({4})
    # without pushdown the selected relations stay in their nodes
    g2 = ghd.choose_ghd(hg, push_selections=False)
    assert sum(n.selection_node for n in g2.nodes()) == 0 and len(g2.nodes()) == 2


def test_fhw_one_is_one_node_and_cyclic_joins_stay_whole():
    star = ghd.Hypergraph(4, [E("F", (0, 1, 2, 3)), E("D3", (2,)), E("D4", (3,))])
    g = ghd.choose_ghd(star)
    assert g.fhw == pytest.approx(1.0) and len(g.nodes()) == 1
    tri = ghd.Hypergraph(3, [E("R", (0, 1)), E("S", (1, 2)), E("T", (0, 2))])
    g = ghd.choose_ghd(tri)
    assert g.fhw == pytest.approx(1.5) and len(g.nodes()) == 1


def test_bowtie_splits_at_the_shared_vertex():
    # two triangles sharing vertex 2: one node costs rho* 3, two nodes 1.5 each
    bow = ghd.Hypergraph(5, [E("a", (0, 1)), E("b", (1, 2)), E("c", (0, 2)), E("d", (2, 3)), E("e", (3, 4)),
                             E("f", (2, 4))])
    g = ghd.choose_ghd(bow)
    assert g.fhw == pytest.approx(1.5)
    assert sorted(sorted(n.bag) for n in g.nodes()) == [[0, 1, 2], [2, 3, 4]]


def test_tie_break_order():
    """Same FHW: fewer nodes first, then depth, then shared vertices, then
    deeper selections (Section 3.2)."""
    hg = ghd.Hypergraph(4, [E("a", (0, 1)), E("b", (1, 2), 1, True), E("c", (2, 3))])
    N = ghd.Node

    def make(tree):
        def rec(t):
            bag, kids = t
            return N(frozenset(bag), [rec(k) for k in kids])
        return ghd.GHD(rec(tree), 1.0)
    one = make(((0, 1, 2, 3), []))
    chain = make(((0, 1), [((1, 2), [((2, 3), [])])]))
    star = make(((1, 2), [((0, 1), []), ((2, 3), [])]))
    assert ghd.ghd_metrics(one, hg) < ghd.ghd_metrics(star, hg)             # fewer nodes
    assert ghd.ghd_metrics(star, hg) < ghd.ghd_metrics(chain, hg)           # same nodes, smaller depth
    wide = make(((0, 1, 2), [((1, 2, 3), [])]))
    narrow = make(((0, 1, 2), [((2, 3), [])]))
    assert ghd.ghd_metrics(narrow, hg) < ghd.ghd_metrics(wide, hg)          # fewer shared vertices
    hg2 = ghd.Hypergraph(4, [E("a", (0, 1)), E("b", (1, 2)), E("c", (2, 3), 1, True)])
    deep = make(((0, 1, 2), [((2, 3), [])]))
    shallow = make(((2, 3), [((0, 1, 2), [])]))
    assert ghd.ghd_metrics(deep, hg2) < ghd.ghd_metrics(shallow, hg2)       # selection lower in the tree


CATALOG = {
    "fact": {"keys": ["f_order", "f_supp"], "columns": ["price", "disc"], "rows": 60},
    "orders": {"keys": ["o_key", "o_cust"], "columns": ["o_date"], "rows": 15},
    "customer": {"keys": ["c_key", "c_nation"], "rows": 5},
    "supplier": {"keys": ["s_key", "s_nation"], "rows": 4},
    "nation": {"keys": ["n_key", "n_region"], "columns": ["n_name"], "rows": 3},
    "region": {"keys": ["r_key"], "columns": ["r_name"], "rows": 2},
}


def test_sql_rules_on_the_bi_query():
    from helpers import BI_QUERY
    tr = sql.translate(BI_QUERY.format(region=2, lo=700, hi=1064), CATALOG)
    # Rule 1: five key vertices (order, customer, nation, supplier, region)
    assert len(tr.vertices) == 5
    v = {(a, k): x for a, _, cols in tr.edges for k, x in cols}
    assert v[("f", "f_order")] == v[("o", "o_key")]
    assert v[("c", "c_nation")] == v[("s", "s_nation")] == v[("n", "n_key")]
    assert v[("n", "n_region")] == v[("r", "r_key")]
    assert len({v[("f", "f_supp")], v[("o", "o_cust")], v[("f", "f_order")], v[("n", "n_key")],
                v[("r", "r_key")]}) == 5
    # Rule 2: no key vertex is an output, all are aggregated away
    assert sorted(tr.alpha) == list(range(5))
    # Rule 3: the aggregated expression annotates fact alone
    assert tr.annotation["f"] is not None and all(tr.annotation[a] is None for a in "ocsnr")
    # Rule 4: the selected and grouped annotations sit in M with their relation
    assert tr.meta == {("r", "r_name"): "r", ("o", "o_date"): "o", ("n", "n_name"): "n"}
    assert [(g[0], g[1].rel, g[1].name) for g in tr.group_by] == [("meta", "n", "n_name")]
    assert sorted((c.rel, c.name, lo, hi) for c, lo, hi in tr.selections) == [("o", "o_date", 700, 1064),
                                                                               ("r", "r_name", 2, 2)]


@pytest.mark.parametrize("text,msg", [
    ("SELECT SUM(f.price * c.c_key) FROM fact f, customer c WHERE f.f_order = c.c_key", "several relations"),
    ("SELECT COUNT(*) FROM fact f, orders o WHERE f.price = o.o_key", "non-key"),
    ("SELECT COUNT(*) FROM fact f WHERE f.nope = 3", "no column"),
    ("SELECT COUNT(*) FROM fact f, orders f", "duplicate alias"),
])
def test_sql_refusals(text, msg):
    with pytest.raises(sql.SQLError) as e:
        sql.translate(text, CATALOG)
    assert msg in str(e.value)


@pytest.mark.parametrize("cond,want", [
    ("o.o_date = 300", (300, 300)),
    ("o.o_date < 300", (-2 ** 31, 299)),
    ("o.o_date <= 300", (-2 ** 31, 300)),
    ("o.o_date > 300", (301, 2 ** 31 - 1)),
    ("o.o_date >= 300", (300, 2 ** 31 - 1)),
    ("o.o_date BETWEEN 10 AND 20", (10, 20)),
])
def test_sql_comparisons_become_inclusive_ranges(cond, want):
    p = sql.parse(f"SELECT COUNT(*) FROM fact f, orders o WHERE f.f_order = o.o_key AND {cond}", CATALOG)
    assert [(c.rel, c.name, lo, hi) for c, lo, hi in p.ranges] == [("o", "o_date") + want]
    assert [(a.rel, a.name, b.rel, b.name) for a, b in p.joins] == [("f", "f_order", "o", "o_key")]


def test_sql_keywords_case_and_unqualified_columns():
    """Keywords in any case, a trailing semicolon, AS aliases in the select
    list and columns without an alias when only one table has them."""
    text = ("select count(*) as n from fact f, orders o "
            "where f_order = o_key and o_date between 5 and 9 group by o_cust;")
    p = sql.parse(text, CATALOG)
    assert p.select == [("count",)]
    assert [(a.rel, a.name, b.rel, b.name) for a, b in p.joins] == [("f", "f_order", "o", "o_key")]
    assert [(c.rel, c.name, lo, hi) for c, lo, hi in p.ranges] == [("o", "o_date", 5, 9)]
    assert [(c.rel, c.name) for c in p.group_by] == [("o", "o_cust")]
    tr = sql.translate(text, CATALOG)
    assert tr.aggregate == ("count",)
    # the grouped key is an output vertex, the joined key is aggregated away
    assert len(tr.vertices) == 2 and len(tr.alpha) == 1


@pytest.mark.parametrize("text,msg", [
    ("SELECT COUNT(*) FROM fact f, orders o WHERE f.f_order <> o.o_key", "unsupported comparison"),
    ("SELECT COUNT(*) FROM fact f, orders o WHERE f.f_order < o.o_key", "only equi-joins"),
    ("SELECT COUNT(*) FROM nowhere n", "unknown table"),
    ("SELECT COUNT(*) FROM fact f WHERE g.f_order = 3", "unknown alias"),
    ("SELECT COUNT(*) FROM fact f GROUP BY f.f_order extra", "unexpected"),
    ("SELECT COUNT(*), SUM(f.price) FROM fact f", "exactly one aggregate"),
    ("SELECT COUNT(*) FROM fact f WHERE f.f_order = 3 $", "cannot read"),
])
def test_sql_more_refusals(text, msg):
    with pytest.raises(sql.SQLError) as e:
        sql.translate(text, CATALOG)
    assert msg in str(e.value)
