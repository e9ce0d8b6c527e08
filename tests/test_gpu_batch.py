"""Batched uneven joins: many triangle / 4-clique COUNT queries in one
persistent, graph-captured launch vs the oracle, per query; replays agree;
the autotuner's pick gives the same counts."""
import math

import numpy as np
import pytest

from helpers import dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu


def make_batch(ctx, lh, graphs, layout=(32, 32)):
    tries, queries = [], []
    for kind, (s, d) in graphs:
        t = ctx.build_trie([dev_u32(s), dev_u32(d)], key_order=[0, 1], layout=layout)
        tries.append(t)
        queries.append((kind, t))
    return tries, queries


def oracle_counts(orc, graphs):
    return np.array([orc.triangle_count(s, d) if k == 0 else orc.clique4_count(s, d) for k, (s, d) in graphs],
                    dtype=np.uint64)


def test_batch_vs_oracle_and_replay(ctx, orc, lhlib):
    lh = lhlib
    ns, ms = gen.batch_graph_sizes(48)
    graphs = []
    for i in range(48):
        m = int(min(ms[i], 20000))
        n = int(max(16, math.ceil(m / 8), math.ceil((1 + math.sqrt(1 + 8 * m)) / 2)))
        graphs.append((i % 2, gen.batch_graph(i, n, m)))
    graphs.append((0, gen.complete_graph(30)))
    graphs.append((1, gen.complete_graph(30)))
    graphs.append((0, gen.chung_lu_edges(20000, 200000, 2.1, 7)))   # hubs: bitset out-sets
    graphs.append((1, gen.chung_lu_edges(3000, 30000, 2.1, 8)))
    want = oracle_counts(orc, graphs)
    assert want[48] == math.comb(30, 3) and want[49] == math.comb(30, 4)
    for layout in ((32, 32), (0, 0)):
        tries, queries = make_batch(ctx, lh, graphs, layout)
        for tuning in (None, (64, 32, 2), (2048, 512, 8)):
            b = lh.Batch(ctx, queries, tuning)
            b.run()
            got1 = b.result()
            b.run()
            got2 = b.result()
            b.free()
            assert np.array_equal(got1, want), (layout, tuning, np.flatnonzero(got1 != want))
            assert np.array_equal(got2, want)
        for t in tries:
            t.free()


def test_autotune_pick_is_exact(ctx, orc, lhlib):
    lh = lhlib
    graphs = [(i % 2, gen.batch_graph(i, 200, 2000)) for i in range(16)]
    want = oracle_counts(orc, graphs)
    tries, queries = make_batch(ctx, lh, graphs)
    tuning, ms = lh.batch_autotune(ctx, queries)
    assert tuning[0] in (64, 256, 2048) and tuning[1] <= tuning[0] and ms > 0
    b = lh.Batch(ctx, queries, tuning)
    b.run()
    assert np.array_equal(b.result(), want)
    b.free()
    for t in tries:
        t.free()


def test_batch_rejects_wrong_trie(ctx, lhlib):
    lh = lhlib
    s, d = gen.complete_graph(10)
    t = ctx.build_trie([dev_u32(s), dev_u32(d)], key_order=[1, 0])
    with pytest.raises(lh.LHError):
        lh.Batch(ctx, [(0, t)])
    t.free()


@pytest.fixture(scope="module")
def full_batch_graphs():
    """The uneven batch at its stated size: 4096 G(n, m) graphs with
    log-uniform edge counts 100..1e5 (even index: triangle, odd: 4-clique)
    plus the 2^24-edge Chung-Lu graph (n = 2^20, exponent 2.1) as one more
    triangle query."""
    graphs = [(i % 2, g) for i, g in enumerate(gen.batch_graphs(4096))]
    graphs.append((0, gen.hub_graph()))
    return graphs


def test_batch_full_size_vs_oracle(ctx, orc, lhlib, full_batch_graphs):
    """Per-query counts of the 4097-query batch equal the oracle's; the hub
    graph's triangles are counted by the oracle over the degree orientation,
    a different route than the id-oriented join the GPU runs."""
    lh = lhlib
    graphs = full_batch_graphs
    want = np.array([orc.triangle_count(s, d) if k == 0 else orc.clique4_count(s, d)
                     for k, (s, d) in graphs[:-1]] + [orc.triangle_count_degree_ordered(*graphs[-1][1])],
                    dtype=np.uint64)
    tries, queries = make_batch(ctx, lh, graphs)
    hub = tries[-1].stats()
    assert hub.level_bs_sets[1] > 0          # hub out-sets took the bitset layout
    tuning, _ = lh.batch_autotune(ctx, queries)
    for tun in (None, tuning):
        b = lh.Batch(ctx, queries, tun)
        b.run()
        got = b.result()
        b.run()
        again = b.result()
        b.free()
        assert np.array_equal(got, want), (tun, np.flatnonzero(got != want)[:10])
        assert np.array_equal(again, want)
    for t in tries:
        t.free()


def test_join_aggregate_batch_mixes_kernel_and_generic_queries(ctx, orc, lhlib):
    """lh_join_aggregate_batch: triangle and 4-clique COUNT queries in the
    identity order share one persistent launch; a 4-cycle, a lollipop and a
    triangle under another order run through the generic driver; every count
    equals the oracle's and the one-by-one lh_join_aggregate's."""
    lh = lhlib
    graphs = [gen.gnm_edges(300 + 100 * i, 2500 + 700 * i, 900 + i) for i in range(3)]
    graphs.append(gen.chung_lu_edges(3000, 30000, 2.1, 904))
    joins, items, want = [], [], []
    for i, (s, d) in enumerate(graphs):
        for shape, order in (("triangle", [0, 1, 2]), ("clique4", [0, 1, 2, 3]), ("cycle4", [0, 1, 2, 3]),
                             ("triangle", [2, 0, 1]), ("lollipop", [0, 2, 1, 3])):
            g = lh.GraphJoin(ctx, dev_u32(s), dev_u32(d), shape)
            joins.append(g)
            plan = lh.make_plan(order)
            tries, q = g._bind(plan, (32, 32))
            items.append((q, plan, tries))
            want.append(orc.GRAPH_COUNT[shape](s, d))
    res = ctx.join_aggregate_batch(items)
    got = [int(r.wait().count) for r in res]
    for r in res:
        r.free()
    one = []
    for q, plan, tries in items:
        r = ctx.join_aggregate(q, plan, tries)
        one.append(int(r.wait().count))
        r.free()
    for g in joins:
        g.free()
    assert got == want
    assert one == want


def test_join_aggregate_batch_empty_and_tuned(ctx, orc, lhlib):
    lh = lhlib
    assert ctx.join_aggregate_batch([]) == []
    s, d = gen.gnm_edges(500, 6000, 910)
    g = lh.GraphJoin(ctx, dev_u32(s), dev_u32(d), "triangle")
    plan = lh.make_plan([0, 1, 2])
    tries, q = g._bind(plan, (32, 32))
    res = ctx.join_aggregate_batch([(q, plan, tries)] * 5, tuning=(64, 32, 2, 0))
    assert [int(r.wait().count) for r in res] == [orc.triangle_count(s, d)] * 5
    for r in res:
        r.free()
    g.free()
