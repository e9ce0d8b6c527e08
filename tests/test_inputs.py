"""The seeded generators that feed both the oracle and the GPU path: the
parallel batch generator returns exactly what the sequential one does."""
import numpy as np

from paper_1708_07859_b300 import inputs as gen


def test_parallel_batch_graphs_equal_sequential():
    par = gen.batch_graphs(80, workers=2)
    seq = gen.batch_graphs(80, workers=1)
    ns, ms = gen.batch_graph_sizes(80)
    assert len(par) == len(seq) == 80
    for i, ((a, b), (c, d)) in enumerate(zip(par, seq)):
        assert np.array_equal(a, c) and np.array_equal(b, d)
        assert a.size == ms[i] and np.all(a < b) and int(b.max()) < ns[i]


def test_chung_lu_has_exactly_m_distinct_oriented_edges():
    s, d = gen.chung_lu_edges(5000, 60000, 2.1, 9)
    assert s.size == 60000 and np.all(s < d)
    assert np.unique(s.astype(np.uint64) * 5000 + d).size == 60000
