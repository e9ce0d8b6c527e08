"""Generic attribute-at-a-time join (Algorithm 1) on the GPU: COUNT of graph
pattern joins vs the oracle, under every attribute order and layout policy
(the result must not depend on the plan)."""
import itertools
import math

import numpy as np
import pytest

from helpers import dev_u32, graph_counts
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu

LAYOUTS = ((0, 0), (32, 32), (8, 8))


def test_triangle_workload_every_order(ctx, orc):
    src, dst = gen.triangle_workload()          # 4096 vertices, 32768 edges
    want = orc.triangle_count(src, dst)
    got = graph_counts(ctx, src, dst, "triangle", list(itertools.permutations(range(3))), LAYOUTS)
    assert set(got.values()) == {want}, (want, got)


@pytest.mark.parametrize("n", [4, 5, 20, 64])
def test_complete_graph_closed_forms(ctx, n):
    s, d = gen.complete_graph(n)
    tri = graph_counts(ctx, s, d, "triangle", [(0, 1, 2), (2, 0, 1)], LAYOUTS)
    assert set(tri.values()) == {math.comb(n, 3)}
    for shape in ("clique4", "cycle4", "lollipop"):
        got = graph_counts(ctx, s, d, shape, [(0, 1, 2, 3), (3, 1, 0, 2)], LAYOUTS)
        assert set(got.values()) == {math.comb(n, 4)}, shape


def test_bipartite_and_wheel(ctx):
    s, d = gen.complete_bipartite(30, 40)
    assert set(graph_counts(ctx, s, d, "triangle", [(0, 1, 2)]).values()) == {0}
    s, d = gen.wheel_graph(50)
    assert set(graph_counts(ctx, s, d, "triangle", [(0, 1, 2), (1, 2, 0)], LAYOUTS).values()) == {50}


@pytest.mark.parametrize("shape", ["clique4", "cycle4", "lollipop"])
def test_four_attribute_patterns_vs_oracle(ctx, orc, shape):
    src, dst = gen.gnm_edges(400, 6000, 77)
    want = orc.GRAPH_COUNT[shape](src, dst)
    orders = [(0, 1, 2, 3), (3, 2, 1, 0), (1, 3, 0, 2), (2, 0, 3, 1)]
    got = graph_counts(ctx, src, dst, shape, orders, LAYOUTS)
    assert set(got.values()) == {want}, (want, got)


def test_every_order_of_cycle4_on_power_law(ctx, orc):
    src, dst = gen.chung_lu_edges(2000, 12000, 2.1, 9)
    want = orc.cycle4_count(src, dst)
    got = graph_counts(ctx, src, dst, "cycle4", list(itertools.permutations(range(4))), ((32, 32),))
    assert set(got.values()) == {want}


@pytest.mark.parametrize("shape", ["path3", "star3"])
def test_acyclic_patterns_vs_algorithm1(ctx, orc, shape):
    src, dst = gen.gnm_edges(30, 90, 5)
    from test_oracle_pins import rels_for
    rels, k = rels_for(shape, src, dst) if shape == "path3" else (
        [{"attrs": a, "tuples": list(zip(src.tolist(), dst.tolist()))} for a in [(0, 1), (0, 2), (0, 3)]], 4)
    want = len(orc.generic_join((0, 1, 2, 3), rels))
    got = graph_counts(ctx, src, dst, shape, [(0, 1, 2, 3), (3, 2, 1, 0), (2, 1, 3, 0)], LAYOUTS)
    assert set(got.values()) == {want}


def test_three_distinct_relations(ctx, orc, lhlib):
    lh = lhlib
    R = gen.gnm_edges(300, 3000, 1)
    S = gen.gnm_edges(300, 3000, 2)
    T = gen.gnm_edges(300, 3000, 3)
    want = orc.join_rst_count(R, S, T)
    dR, dS, dT = [[dev_u32(x) for x in r] for r in (R, S, T)]
    q = lh.make_query(3, [{"slot": 0, "attrs": [0, 1], "card": 3000},
                          {"slot": 1, "attrs": [1, 2], "card": 3000},
                          {"slot": 2, "attrs": [0, 2], "card": 3000}])
    for order in itertools.permutations(range(3)):
        plan = lh.make_plan(list(order))
        tries = []
        for e, rel in enumerate((dR, dS, dT)):
            tries.append(ctx.build_trie(rel, key_order=ctx.edge_key_order(q, plan, e)))
        r = ctx.join_aggregate(q, plan, tries)
        assert r.wait().count == want, order
        r.free()
        for t in tries:
            t.free()


def test_wrong_trie_order_is_rejected(ctx, lhlib):
    lh = lhlib
    s, d = gen.complete_graph(6)
    ds, dd = dev_u32(s), dev_u32(d)
    q = lh.make_query(2, [{"slot": 0, "attrs": [0, 1], "card": 15}])
    fwd = ctx.build_trie([ds, dd], key_order=[0, 1])
    with pytest.raises(lh.LHError) as e:
        ctx.join_aggregate(q, lh.make_plan([1, 0]), [fwd])
    assert e.value.status == lh.EINVAL
    r = ctx.join_aggregate(q, lh.make_plan([0, 1]), [fwd])
    assert r.wait().count == 15
    r.free()
    fwd.free()


PAIR_LAYOUTS = ((0, 0), (32, 32), (8, 8), (128, 128))


@pytest.mark.parametrize("shape", ["triangle", "cycle4", "lollipop"])
def test_last_attribute_pair_count_matches_probe_and_oracle(ctx, orc, shape):
    """The count-only pair path at the last attribute (merge path, or scans
    probing a bitset / searching a uint set, in work items spread over
    warps) against the one-thread-per-candidate probe path and the oracle,
    on a power-law graph whose hub sets take every layout."""
    from paper_1708_07859_b300 import lh
    src, dst = gen.chung_lu_edges(5000, 60000, 2.1, 31)
    want = orc.GRAPH_COUNT[shape](src, dst)
    n_attrs = 3 if shape == "triangle" else 4
    orders = [tuple(range(n_attrs)), tuple(reversed(range(n_attrs)))]
    auto = graph_counts(ctx, src, dst, shape, orders, PAIR_LAYOUTS, isect_impl=lh.ISECT_AUTO)
    probe = graph_counts(ctx, src, dst, shape, orders, PAIR_LAYOUTS, isect_impl=lh.ISECT_PROBE)
    assert set(auto.values()) == {want}, (want, auto)
    assert set(probe.values()) == {want}, (want, probe)


@pytest.mark.parametrize("n", [33, 97, 300])
def test_last_attribute_pair_count_on_complete_graphs(ctx, n):
    """K_n: every set of the last attribute is a contiguous run, so uint
    layouts merge and bitset layouts probe; sizes straddle the 32-element
    threshold of the pair path."""
    s, d = gen.complete_graph(n)
    got = graph_counts(ctx, s, d, "triangle", [(0, 1, 2), (2, 1, 0)], PAIR_LAYOUTS)
    assert set(got.values()) == {math.comb(n, 3)}
    got = graph_counts(ctx, s, d, "cycle4", [(0, 1, 2, 3)], ((0, 0), (32, 32)))
    assert set(got.values()) == {math.comb(n, 4)}


def test_pair_item_list_overflow_keeps_counts_exact(ctx):
    """K_3000 triangles (4.5M edges): a last-attribute chunk of 2^22 entries
    asks for more work items than the list holds, so some entries fall back
    to the probe path within the same launch; the count stays C(3000, 3)."""
    s, d = gen.complete_graph(3000)
    got = graph_counts(ctx, s, d, "triangle", [(0, 1, 2)], ((0, 0), (32, 32)))
    assert set(got.values()) == {math.comb(3000, 3)}


def test_visited_counts_pair_path_reads(ctx, lhlib):
    """`visited` includes the elements the pair path reads (a triangle query
    on K_200 sends every large last-attribute pair there)."""
    s, d = gen.complete_graph(200)
    out = {}
    for impl in (lhlib.ISECT_AUTO, lhlib.ISECT_PROBE):
        g = lhlib.GraphJoin(ctx, dev_u32(s), dev_u32(d), "triangle", isect_impl=impl)
        plan = lhlib.make_plan([0, 1, 2], bs_ratio=0)
        tries, q = g._bind(plan, (0, 0))
        r = ctx.join_aggregate(q, plan, tries)
        v = r.wait()
        out[impl] = (int(v.count), int(v.visited))
        r.free()
        g.free()
    assert out[lhlib.ISECT_AUTO][0] == out[lhlib.ISECT_PROBE][0] == math.comb(200, 3)
    assert out[lhlib.ISECT_AUTO][1] > 0 and out[lhlib.ISECT_PROBE][1] > 0
