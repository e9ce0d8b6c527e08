"""Failure handling without a GPU fault: bounded device waits report
LH_ETIMEOUT and leave the context usable; host-side time budgets stop a
join; bad arguments are refused before any launch."""
import numpy as np
import pytest

from helpers import dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(ctx, orc, lhlib):
    lh = lhlib
    st = lh.lib().lh_selftest_bounded_wait(ctx.h, 2000)
    assert st == lh.ETIMEOUT
    ctx.sync()  # the status word was consumed; nothing pending
    s, d = gen.gnm_edges(200, 1500, 3)
    got = lh.GraphJoin(ctx, dev_u32(s), dev_u32(d), "triangle")
    assert got.run(lh.make_plan([0, 1, 2]))[0] == orc.triangle_count(s, d)
    got.free()


def test_plan_time_budget_reports_timeout(ctx, lhlib):
    lh = lhlib
    s, d = gen.chung_lu_edges(20000, 300000, 2.0, 5)
    g = lh.GraphJoin(ctx, dev_u32(s), dev_u32(d), "cycle4")
    # a 0.001 ms budget is exceeded by any multi-chunk run: the call reports
    # the budget instead of a time, and the context stays usable
    assert g.time_plan(lh.make_plan([3, 2, 1, 0]), budget_ms=0.001) is None
    assert g.time_plan(lh.make_plan([0, 1, 2, 3]), budget_ms=0.0) > 0
    g.free()


def test_bad_arguments_are_refused(ctx, lhlib):
    lh = lhlib
    assert lh.lib().lh_selftest_bounded_wait(ctx.h, 0) == lh.EINVAL
    s, d = gen.complete_graph(5)
    t = ctx.build_trie([dev_u32(s), dev_u32(d)])
    q = lh.make_query(3, [{"slot": 0, "attrs": [0, 1], "card": 10}])
    with pytest.raises(lh.LHError) as e:       # attribute 2 is in no relation
        ctx.join_aggregate(q, lh.make_plan([0, 1, 2]), [t])
    assert e.value.status == lh.EINVAL
    with pytest.raises(lh.LHError):
        ctx.build_trie([dev_u32(s), dev_u32(d)], key_order=[0, 0])
    t.free()


def test_pool_reserve_and_refusal(ctx, orc, lhlib):
    """A reservation maps memory into the context's pool; one the device
    cannot provide is refused with LH_ENOMEM (an allocation error, not a
    fault) and the context goes on working."""
    lh = lhlib
    ctx.pool_reserve(64 << 20)
    with pytest.raises(lh.LHError) as e:
        ctx.pool_reserve(1 << 50)
    assert e.value.status == lh.ENOMEM
    s, d = gen.gnm_edges(300, 2000, 4)
    g = lh.GraphJoin(ctx, dev_u32(s), dev_u32(d), "triangle")
    assert g.run(lh.make_plan([0, 1, 2]))[0] == orc.triangle_count(s, d)
    g.free()


@pytest.mark.parametrize("bad", [100, -1])
def test_group_value_outside_its_domain_is_refused(ctx, orc, lhlib, bad):
    """A GROUP BY value at or above its declared card (or a negative int32)
    is reported as LH_EINVAL when the result is waited on, instead of being
    merged into some group; the context keeps working."""
    import torch
    from helpers import dev
    lh = lhlib
    data = gen.star_schema(20_000, dims=(300, 80, 30, 5), seed=23)
    data["d3_grp"] = data["d3_grp"].copy()
    data["d3_grp"][int(data["k"][2][0])] = bad          # the first fact row's group leaves [0, 100)
    keys = [dev_u32(k) for k in data["k"]]
    sj = lh.StarJoin(ctx, keys, dev(data["price"]), dev(data["disc"]), dev(data["d3_grp"]),
                     dev(data["d4_region"]))
    t1 = ctx.filter_trie(dev(data["d1_date"]), 0, 10_000)
    t2 = ctx.filter_trie(dev(data["d2_cat"]), 0, 100)
    with pytest.raises(lh.LHError) as e:
        sj.run(t1, t2)
    assert e.value.status == lh.EINVAL
    ctx.sync()
    s, d = gen.gnm_edges(200, 1500, 3)
    g = lh.GraphJoin(ctx, dev_u32(s), dev_u32(d), "triangle")
    assert g.run(lh.make_plan([0, 1, 2]))[0] == orc.triangle_count(s, d)
    g.free(); t1.free(); t2.free(); sj.free()
