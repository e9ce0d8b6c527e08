"""Kernel tracing: every launch is counted while tracing is on; with a
kernel name given, only that kernel is bracketed by events."""
import numpy as np
import pytest

from helpers import dev, dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu


def build(ctx, lh):
    r, c, v = gen.uniform_coo(3000, 2000, 12, 77)
    return lh.matrix_trie(ctx, dev_u32(r), dev_u32(c), dev(v))


def test_trace_counts_every_launch_and_times_the_named_kernel(ctx, lhlib):
    lh = lhlib
    ctx.trace_reset()
    ctx.trace_only(None)
    ctx.trace(True)
    build(ctx, lh).free()
    ctx.trace(False)
    full = ctx.trace_read()
    assert "k_sort_onesweep" in full and "k_levels" in full
    assert all(ms > 0 for _, ms in full.values())

    ctx.trace_reset()
    ctx.trace_only("k_levels")
    ctx.trace(True)
    build(ctx, lh).free()
    ctx.trace(False)
    ctx.trace_only(None)
    only = ctx.trace_read()
    # the same launches are counted; only k_levels carries event time
    assert {k: n for k, (n, _) in only.items()} == {k: n for k, (n, _) in full.items()}
    assert only["k_levels"][1] > 0
    assert all(ms == 0 for k, (_, ms) in only.items() if k != "k_levels")
