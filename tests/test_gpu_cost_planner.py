"""The library's Section 4 cost model (lh_plan with LH_PLANNER_COST and
lh_plan_explain) against the oracle's restatement of it, on the paper's two
printed examples and on random query hypergraphs.

The library's copy (icost fold, score, weight, candidate orders, the
Section 4.1.2 relaxation, lexicographic ties) is C++ inside liblh; the
oracle's is plain Python pinned to the printed values in
tests/golden/q5_cost_example.json.  Both must agree exactly: the cost model
is integer arithmetic."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_q5():
    with open(os.path.join(GOLDEN, "q5_cost_example.json")) as f:
        return json.load(f)


def query_of(lh, n_attrs, rel_attrs, cards, materialized=(), eq_selected=(), dense=()):
    edges = []
    for e, (attrs, card) in enumerate(zip(rel_attrs, cards)):
        edges.append({"slot": -1 if e in dense else e, "attrs": list(attrs), "card": int(card)})
    return lh.make_query(n_attrs, edges, materialized=materialized, eq_selected=eq_selected)


def test_q5_node_printed_icosts_weights_and_cost(ctx, orc, lhlib):
    """Section 4.1.1 / 4.2 example: order [orderkey, custkey, nationkey,
    suppkey] has icosts (1, 10, 11, 50) and weights (26, 3, 1, 1)."""
    g = load_q5()
    verts = g["vertices"]
    vid = {v: i for i, v in enumerate(verts)}
    rels = ["lineitem", "orders", "customer", "supplier", "nation"]
    rel_attrs = [tuple(vid[a] for a in g["relations"][r]) for r in rels]
    heavy = g["score_derived"]["heavy"]
    # lineitem and orders from the printed trie census; the three small
    # relations take cardinalities that reproduce their printed scores
    # (score 3: a card in (2%, 3%] of lineitem's; score 1: at most 1%)
    cards = [heavy, g["score_derived"]["card"], int(0.028 * heavy), int(0.004 * heavy), 30]
    q = query_of(lhlib, len(verts), rel_attrs, cards)
    order = [vid[v] for v in g["order"]]
    ic, w, cost = ctx.plan_explain(q, order)
    assert ic == g["icost_printed"]
    assert {verts[a]: w[a] for a in range(len(verts))} == g["weights_printed"]
    assert cost == g["cost_derived"]
    # and the oracle's copy on the same query
    ow = orc.weights(rel_attrs, cards)
    assert orc.icosts(tuple(order), rel_attrs) == ic
    assert [ow[a] for a in range(len(verts))] == w
    assert orc.cost(tuple(order), rel_attrs, ow) == cost
    # the planner's argmin over every order equals the oracle's
    p = ctx.plan(q)
    o_order, o_cost = orc.best_order(list(range(len(verts))), rel_attrs, cards)
    assert p.order_list() == list(o_order) and p.cost == o_cost


def test_smm_example_icosts_and_relaxed_order(ctx, orc, lhlib):
    """Section 4.1.2 example, M1(i,k) M2(k,j) with k projected away: the
    icost of k is 50 in order [i, j, k] and 10 in [i, k, j], and the
    relaxation picks [i, k, j]."""
    smm = load_q5()["smm"]
    i, k, j = 0, 1, 2
    rel_attrs = [(i, k), (k, j)]
    cards = [100, 100]
    q = query_of(lhlib, 3, rel_attrs, cards, materialized=(i, j))
    ic, _, _ = ctx.plan_explain(q, [i, j, k])
    assert ic[2] == smm["icost_k_order_ijk"]
    ic, _, _ = ctx.plan_explain(q, [i, k, j])
    assert ic[1] == smm["icost_k_order_ikj"]
    p = ctx.plan(q)
    o_order, o_cost = orc.best_order([i, j, k], rel_attrs, cards, materialized={i, j})
    assert p.order_list() == [i, k, j] == list(o_order)
    assert p.cost == o_cost


def random_hypergraph(rng):
    n_attrs = int(rng.integers(2, 6))
    n_edges = int(rng.integers(2, 6))
    rel_attrs = []
    for _ in range(n_edges):
        ar = int(rng.integers(1, min(3, n_attrs) + 1))
        rel_attrs.append(tuple(int(a) for a in rng.choice(n_attrs, size=ar, replace=False)))
    # every attribute in at least one relation
    for a in range(n_attrs):
        if not any(a in r for r in rel_attrs):
            rel_attrs[int(rng.integers(0, n_edges))] += (a,)
    rel_attrs = [tuple(r[:6]) for r in rel_attrs]
    # cardinalities spread over orders of magnitude (scores from 1 to 100),
    # with ties now and then
    cards = [int(10 ** rng.uniform(1, 8)) for _ in range(n_edges)]
    if rng.random() < 0.3:
        cards[1] = cards[0]
    mat = tuple(int(a) for a in range(n_attrs) if rng.random() < 0.5)
    eq = tuple(int(a) for a in range(n_attrs) if rng.random() < 0.25)
    dense = tuple(e for e in range(n_edges) if len(rel_attrs[e]) == 1 and rng.random() < 0.3)
    return n_attrs, rel_attrs, cards, mat, eq, dense


@pytest.mark.parametrize("seed", range(50))
def test_random_hypergraphs_match_oracle(ctx, orc, lhlib, seed):
    rng = np.random.default_rng(1000 + seed)
    n_attrs, rel_attrs, cards, mat, eq, dense = random_hypergraph(rng)
    q = query_of(lhlib, n_attrs, rel_attrs, cards, materialized=mat, eq_selected=eq, dense=dense)
    p = ctx.plan(q)
    o_order, o_cost = orc.best_order(list(range(n_attrs)), rel_attrs, cards, materialized=set(mat),
                                     eq_selected=set(eq), dense=set(dense))
    assert p.order_list() == list(o_order), (rel_attrs, cards, mat, eq, dense)
    assert p.cost == o_cost
    assert p.n_candidates == len(orc.candidate_orders(list(range(n_attrs)), set(mat), rel_attrs, set(dense)))
    # every order's terms, not only the argmin's
    w = orc.weights(rel_attrs, cards, set(eq))
    for o in orc.candidate_orders(list(range(n_attrs)), set(mat), rel_attrs, set(dense))[:12]:
        ic, lw, c = ctx.plan_explain(q, list(o))
        assert ic == orc.icosts(o, rel_attrs, set(dense))
        assert lw == [w[a] for a in range(n_attrs)]
        assert c == orc.cost(o, rel_attrs, w, set(dense))
