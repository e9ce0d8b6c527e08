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


def test_planner_training_graphs_are_held_out_from_its_evaluation():
    """The learned planner's training graphs (10K queries: 1667 graphs, six
    templates each) are drawn from seeds disjoint from the evaluation graphs'
    and stay at or below 2^20 edges, while the evaluation graphs have 2^22:
    the trained model is evaluated on graphs it never saw."""
    from paper_1708_07859_b300 import planner
    n_graphs = (10000 + len(planner.TEMPLATES) - 1) // len(planner.TEMPLATES)
    seeds = np.random.default_rng(planner.TRAIN_SEED).integers(0, 2 ** 31, size=n_graphs)
    eval_seeds = {planner.EVAL_SEED + i for i in range(5)}
    assert not (set(int(x) for x in seeds) & eval_seeds)
    # the graphs the first training seeds yield stay within [2^10, 2^20] edges
    for x in seeds[:3]:
        (src, dst), desc = planner.random_graph(np.random.default_rng(int(x)))
        assert 2 ** 10 <= src.size <= 2 ** 20 and desc[2] == src.size
    s, d = gen.chung_lu_edges(1 << 12, 1 << 14, 2.1, planner.EVAL_SEED)   # the evaluation generator, small
    assert s.size == 1 << 14 and np.all(s < d)
