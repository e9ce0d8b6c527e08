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
