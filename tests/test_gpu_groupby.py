"""GROUP BY on annotations of any width (Section 5) on the GPU: dense group
arrays, per-warp private tables and the shared concurrent table give the
oracle's groups -- key tuples exact, counts exact, sums within 1e-6 of the
fp64 oracle -- and the automatic choice follows the paper's width rule."""
import numpy as np
import pytest

from helpers import dev, dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu

REL_TOL = 1e-6
COLS = {0: "d1_seg", 1: "d2_cat", 2: "d3_grp", 3: "d4_region"}
CARDS = {0: 5, 1: 40, 2: 100, 3: 5}


@pytest.fixture(scope="module")
def star(ctx, lhlib):
    lh = lhlib
    data = gen.star_schema(400_000, dims=(20_000, 4_000, 1_000, 25), seed=31)
    keys = [dev_u32(k) for k in data["k"]]
    dims = {i: dev(data[c]) for i, c in COLS.items()}
    sj = lh.StarJoin(ctx, keys, dev(data["price"]), dev(data["disc"]), dim_cols=dims, dim_cards=CARDS)
    f1, f2 = gen.date_range_for_selectivity(0.2), (0, 19)
    t1 = ctx.filter_trie(dev(data["d1_date"]), *f1)
    t2 = ctx.filter_trie(dev(data["d2_cat"]), *f2)
    yield lh, data, sj, t1, t2, f1, f2
    t1.free(); t2.free(); sj.free()


def check(keys, gs, gc, wk, ws, wc):
    o = np.lexsort(keys.T[::-1])
    keys, gs, gc = keys[o], gs[o], gc[o]
    assert np.array_equal(keys, wk)
    assert np.array_equal(gc, wc)
    err = np.abs(gs - ws)
    assert np.all(err <= REL_TOL * np.abs(ws) + 1e-9), float(np.max(err / np.abs(ws)))


@pytest.mark.parametrize("groups", [(2, 3), (1, 2, 3), (0, 1, 2, 3), (3, 2, 1, 0)])
@pytest.mark.parametrize("impl", ["private", "shared"])
def test_hash_group_by_matches_oracle(orc, star, groups, impl):
    lh, data, sj, t1, t2, f1, f2 = star
    gi = {"private": lh.GROUP_PRIVATE, "shared": lh.GROUP_SHARED}[impl]
    gs, gc, v, keys = sj.run(t1, t2, groups=groups, group_impl=gi, keys=True)
    assert v.group_impl == gi and v.n_group_cols == len(groups)
    wk, ws, wc = orc.star_sum_keys(data, f1, f2, [(d, COLS[d]) for d in groups])
    check(keys, gs, gc, wk, ws, wc)


def test_auto_choice_follows_the_width_rule(orc, star):
    """Two declared columns with a small domain: dense arrays; three: the
    private tables; four (wider than three values): the shared table; three
    undeclared 32-bit columns (96 bits, no packed key): the shared table."""
    lh, data, sj, t1, t2, f1, f2 = star
    for groups, cards, want in (((2, 3), True, lh.GROUP_DENSE), ((1, 2, 3), True, lh.GROUP_PRIVATE),
                                ((0, 1, 2, 3), True, lh.GROUP_SHARED), ((1, 2, 3), False, lh.GROUP_SHARED)):
        gs, gc, v, keys = sj.run(t1, t2, groups=groups, cards=cards, keys=True)
        assert v.group_impl == want, (groups, cards)
        wk, ws, wc = orc.star_sum_keys(data, f1, f2, [(d, COLS[d]) for d in groups])
        if want == lh.GROUP_DENSE:
            g = wk[:, 0].astype(np.int64) * CARDS[groups[1]] + wk[:, 1]
            assert np.array_equal(gc[g], wc) and int(gc.sum()) == int(wc.sum())
            assert np.all(np.abs(gs[g] - ws) <= REL_TOL * ws)
        else:
            check(keys, gs, gc, wk, ws, wc)


def test_private_tables_spill_when_full(orc, star):
    """A warp table holds 256 groups; 4-column keys over this data have
    thousands of groups, so private tables overflow into the shared table and
    the totals still match."""
    lh, data, sj, t1, t2, f1, f2 = star
    gs, gc, v, keys = sj.run(t1, t2, groups=(0, 1, 2, 3), group_impl=lh.GROUP_PRIVATE, keys=True)
    wk, ws, wc = orc.star_sum_keys(data, f1, f2, [(d, COLS[d]) for d in (0, 1, 2, 3)])
    assert wk.shape[0] > 1000
    check(keys, gs, gc, wk, ws, wc)


def test_full_shared_table_is_reported(ctx, orc, star):
    lh, data, sj, t1, t2, f1, f2 = star
    with pytest.raises(lh.LHError) as e:
        sj.run(t1, t2, groups=(0, 1, 2, 3), group_impl=lh.GROUP_SHARED, group_capacity=64)
    assert e.value.status == lh.EOVERFLOW
    ctx.sync()
    gs, gc, v = sj.run(t1, t2)                          # the context keeps working
    ws, wc = orc.star_sum(data, f1, f2)
    assert np.array_equal(gc, wc)


def test_dense_refused_for_undeclared_domains(star):
    lh, data, sj, t1, t2, f1, f2 = star
    with pytest.raises(lh.LHError) as e:
        sj.run(t1, t2, groups=(2, 3), group_impl=lh.GROUP_DENSE, cards=False)
    assert e.value.status == lh.EUNSUPPORTED
