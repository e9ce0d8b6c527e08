"""Multi-node GHD plans with selections pushed into nodes of their own
(Sections 2.3, 3.2) on the six-relation BI query, from SQL text (Section
3.1) through the C ABI: per-group sums within 1e-6 of the fp64 pairwise-join
oracle and exact counts, with and without the pushdown and as one node."""
import numpy as np
import pytest

from helpers import BI_QUERY, bi_catalog
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu

SMALL = {"fact": 2_000_000, "orders": 500_000, "customer": 50_000, "supplier": 5_000, "nation": 25, "region": 5}


@pytest.fixture(scope="module")
def bi(ctx):
    data = gen.bi_schema(SMALL, seed=41)
    return data, bi_catalog(data)


def check(out, orc, data, region, dates):
    ws, wc = orc.bi_q5(data, region, dates)
    want = {(g,): (float(ws[g]), int(wc[g])) for g in np.flatnonzero(wc)}
    assert sorted(out) == sorted(want)
    for k, (s, c) in out.items():
        assert c == want[k][1]
        assert abs(s - want[k][0]) <= 1e-6 * abs(want[k][0])


@pytest.mark.parametrize("pushdown", [True, False])
@pytest.mark.parametrize("region,dates", [(2, (700, 1064)), (0, (0, 2556)), (4, (100, 130))])
def test_bi_query_two_node_ghd(ctx, orc, lhlib, bi, pushdown, region, dates):
    from paper_1708_07859_b300 import sql
    data, cat = bi
    text = BI_QUERY.format(region=region, lo=dates[0], hi=dates[1])
    out, tr, plan = sql.plan_and_run(ctx, text, cat, pushdown=pushdown)
    # the paper's plan: a root over the four-cycle of keys and one child
    # over (nation, region); with the pushdown the region and orders
    # selections sit in nodes of their own
    root = plan.root
    assert plan.fhw == 2.0 and len(root.bag) == 4
    inner = [c for c in root.children if not c.selection_node]
    assert len(inner) == 1 and len(inner[0].bag) == 2
    sel_nodes = [n for n in plan.nodes() if n.selection_node]
    assert len(sel_nodes) == (2 if pushdown else 0)
    check(out, orc, data, region, dates)


def test_bi_query_as_one_node(ctx, orc, lhlib, bi):
    """The same query as a single worst-case optimal join (every relation
    and the selections' filter relations in one node) gives the same groups."""
    from paper_1708_07859_b300 import ghd, sql
    data, cat = bi
    text = BI_QUERY.format(region=2, lo=700, hi=1064)
    out, tr, plan = sql.plan_and_run(ctx, text, cat, pushdown=False, single_node=True)
    assert len(plan.nodes()) == 1
    check(out, orc, data, 2, (700, 1064))
