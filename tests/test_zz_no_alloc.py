"""The allocation-free intersection entry point gives the same counts as the
allocating one.

lh_intersect_count_batch_noalloc serves callers that cannot allocate device
memory while they run queries (an application whose allocator owns the
GPU's memory, or a latency-bound loop).  It keeps its scratch in one fixed
device array shared by every call, so this test calls it twice in a row --
a large batch, then a smaller, different one -- and checks each against the
ordinary entry point through the C ABI.  Counts are integers: they must be
equal.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu


def _bitset(vals):
    v = np.asarray(vals, dtype=np.uint64)
    base = int(v[0]) & ~127
    nw = (((int(v[-1]) - base) >> 5) + 1 + 3) & ~3
    words = np.zeros(nw, dtype=np.uint32)
    d = v - base
    np.bitwise_or.at(words, (d >> 5).astype(np.int64), np.uint32(1) << (d & 31).astype(np.uint32))
    return base, words


def _batch(lh, seed, npairs):
    """Device lh_set arrays for npairs pairs mixing every layout pairing."""
    import torch
    rng = np.random.default_rng(seed)
    keep, da, db = [], [], []
    for p in range(npairs):
        span = int(rng.integers(1000, 400000))
        ca = int(rng.integers(0, span // 2))
        cb = int(rng.integers(1, span // 2))
        sets = [gen.sorted_set(ca, span, seed * 100000 + 2 * p) if ca else np.zeros(0, np.uint32),
                gen.sorted_set(cb, span, seed * 100000 + 2 * p + 1)]
        for side, vals in enumerate(sets):
            layout = int(rng.integers(0, 2)) if vals.size else 0
            if layout == 1:
                base, words = _bitset(vals)
                t = lh.to_device_u32(words)
                d = (1, base, words.size, t.data_ptr())
            else:
                t = lh.to_device_u32(vals if vals.size else np.zeros(1, np.uint32))
                d = (0, 0, vals.size, t.data_ptr())
            keep.append(t)
            (da if side == 0 else db).append(d)
    A = torch.frombuffer(bytearray(lh.pack_sets(da)), dtype=torch.uint8).cuda()
    B = torch.frombuffer(bytearray(lh.pack_sets(db)), dtype=torch.uint8).cuda()
    return A, B, keep


def test_noalloc_matches_allocating_entry_point_twice(ctx, lhlib):
    import torch
    lh = lhlib
    for seed, npairs in ((1, 300), (2, 37)):
        A, B, keep = _batch(lh, seed, npairs)
        want = torch.zeros(npairs, dtype=torch.int64, device="cuda")
        got = torch.full((npairs,), -1, dtype=torch.int64, device="cuda")
        ctx.intersect_count_batch(A, B, want)
        ctx.intersect_count_batch_noalloc(A, B, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want), seed


def test_noalloc_rejects_batches_above_its_limit(ctx, lhlib):
    import torch
    lh = lhlib
    A, B, keep = _batch(lh, 3, 2)
    counts = torch.full((2,), 7, dtype=torch.int64, device="cuda")
    with pytest.raises(lh.LHError) as e:
        ctx.intersect_count_batch_noalloc(A, B, counts, npairs=65537)
    assert e.value.status == lh.EINVAL and "65536" in str(e.value)
    assert counts.tolist() == [7, 7]
