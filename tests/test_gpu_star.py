"""Star-schema BI join-aggregate on the GPU: SUM(price * (1 - discount))
with pushed-down range selections and GROUP BY two dimension attributes,
fp32-compensated per CTA with fp64 group totals, vs the fp64 oracle
(per-group relative error <= 1e-6, counts exact)."""
import numpy as np
import pytest

from helpers import dev, dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


def run_star(ctx, lh, data, f1, f2, order=(0, 1, 2, 3)):
    keys = [dev_u32(k) for k in data["k"]]
    sj = lh.StarJoin(ctx, keys, dev(data["price"]), dev(data["disc"]), dev(data["d3_grp"]),
                     dev(data["d4_region"]))
    t1 = ctx.filter_trie(dev(data["d1_date"]), *f1)
    t2 = ctx.filter_trie(dev(data["d2_cat"]), *f2)
    try:
        gs, gc, v = sj.run(t1, t2, order)
    finally:
        t1.free(); t2.free(); sj.free()
    return gs, gc


def check(gs, gc, ws, wc):
    assert np.array_equal(gc, wc)
    err = np.abs(gs - ws)
    assert np.all(err <= REL_TOL * np.abs(ws) + 1e-9), float(np.max(err / np.maximum(np.abs(ws), 1e-30)))


@pytest.mark.parametrize("sel", [0.01, 0.2, 1.0])
def test_star_small(ctx, orc, lhlib, sel):
    data = gen.star_schema(50_000, dims=(3000, 800, 300, 25), seed=21)
    f1 = gen.date_range_for_selectivity(sel)
    f2 = (0, 7)
    gs, gc = run_star(ctx, lhlib, data, f1, f2)
    ws, wc = orc.star_sum(data, f1, f2)
    check(gs, gc, ws, wc)


def test_star_empty_filter(ctx, orc, lhlib):
    data = gen.star_schema(10_000, dims=(300, 80, 30, 5), seed=22)
    gs, gc = run_star(ctx, lhlib, data, (5000, 6000), (0, 7))
    assert gc.sum() == 0 and np.all(gs == 0)


@pytest.fixture(scope="module")
def full_star(ctx, lhlib):
    """The 60M-row fact trie (dims 1.5M/200K/10K/25) built once for the
    full-size selectivities."""
    lh = lhlib
    data = gen.star_schema()
    keys = [dev_u32(k) for k in data["k"]]
    sj = lh.StarJoin(ctx, keys, dev(data["price"]), dev(data["disc"]), dev(data["d3_grp"]),
                     dev(data["d4_region"]))
    d1, d2 = dev(data["d1_date"]), dev(data["d2_cat"])
    yield data, sj, d1, d2
    sj.free()


@pytest.mark.parametrize("sel", [0.01, 0.05, 0.2])
def test_star_full_size(ctx, orc, lhlib, full_star, sel):
    data, sj, d1, d2 = full_star
    f1 = gen.date_range_for_selectivity(sel)
    f2 = (0, 7)
    t1 = ctx.filter_trie(d1, *f1)
    t2 = ctx.filter_trie(d2, *f2)
    try:
        gs, gc, _ = sj.run(t1, t2)
    finally:
        t1.free(); t2.free()
    ws, wc = orc.star_sum(data, f1, f2)
    check(gs, gc, ws, wc)
    assert gc.sum() > 0
