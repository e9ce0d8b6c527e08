"""The allocation-free intersection entry point gives the same counts as the
allocating one, and as the oracle.

lh_intersect_count_batch_noalloc serves callers that cannot allocate device
memory while they run queries (an application whose allocator owns the
GPU's memory, or a latency-bound loop).  It keeps its scratch in one fixed
device array shared by every call, so the first test calls it twice in a
row -- a large batch, then a smaller, different one -- and checks each
against the ordinary entry point through the C ABI and against the CPU
oracle's plain merge.  Larger batches cover the single-block scan of tile
counts across many 1024-pair chunks, up to the 65536-pair limit itself.
Counts are integers: they must be equal.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu

LIMIT = 65536


def _bitset(vals):
    v = np.asarray(vals, dtype=np.uint64)
    base = int(v[0]) & ~127
    nw = (((int(v[-1]) - base) >> 5) + 1 + 3) & ~3
    words = np.zeros(nw, dtype=np.uint32)
    d = v - base
    np.bitwise_or.at(words, (d >> 5).astype(np.int64), np.uint32(1) << (d & 31).astype(np.uint32))
    return base, words


def _batch(lh, seed, npairs, span_range=(1000, 400000), tiny=False):
    """Device lh_set arrays for npairs pairs mixing every layout pairing, all
    sets packed into one device buffer (16-byte aligned per set); returns the
    two lh_set arrays, the buffer and the sets' values for the oracle."""
    import torch
    rng = np.random.default_rng(seed)
    chunks, descs, vals_of = [], [[], []], [[], []]
    at = 0
    for p in range(npairs):
        span = int(rng.integers(*span_range))
        if tiny:
            ca, cb = int(rng.integers(0, 9)), int(rng.integers(1, 9))
        else:
            ca, cb = int(rng.integers(0, span // 2)), int(rng.integers(1, span // 2))
        sets = [gen.sorted_set(ca, span, seed * 1000003 + 2 * p) if ca else np.zeros(0, np.uint32),
                gen.sorted_set(cb, span, seed * 1000003 + 2 * p + 1)]
        for side, vals in enumerate(sets):
            layout = int(rng.integers(0, 2)) if vals.size else 0
            if layout == 1:
                base, data = _bitset(vals)
                n = data.size
            else:
                base, data, n = 0, vals, vals.size
            pad = (-data.size) % 4
            chunks.append(np.concatenate([data, np.zeros(pad + (4 if data.size == 0 else 0), np.uint32)]))
            descs[side].append((layout, base, n, at))
            vals_of[side].append(vals)
            at += chunks[-1].size
    buf = lh.to_device_u32(np.concatenate(chunks))
    ptr = buf.data_ptr()
    packed = [lh.pack_sets([(l, b, n, ptr + 4 * off) for (l, b, n, off) in d]) for d in descs]
    A = torch.frombuffer(bytearray(packed[0]), dtype=torch.uint8).cuda()
    B = torch.frombuffer(bytearray(packed[1]), dtype=torch.uint8).cuda()
    return A, B, buf, vals_of


def _oracle_counts(orc, vals_of):
    return np.array([orc.intersect_count(a, b) for a, b in zip(*vals_of)], dtype=np.int64)


def _check(ctx, orc, lh, A, B, vals_of, npairs):
    import torch
    want = torch.zeros(npairs, dtype=torch.int64, device="cuda")
    got = torch.full((npairs,), -1, dtype=torch.int64, device="cuda")
    ctx.intersect_count_batch(A, B, want)
    ctx.intersect_count_batch_noalloc(A, B, got)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    assert np.array_equal(got.cpu().numpy(), _oracle_counts(orc, vals_of))


def test_noalloc_matches_allocating_entry_point_twice(ctx, orc, lhlib):
    for seed, npairs in ((1, 300), (2, 37)):
        A, B, buf, vals_of = _batch(lhlib, seed, npairs)
        _check(ctx, orc, lhlib, A, B, vals_of, npairs)


def test_noalloc_many_tiny_pairs(ctx, orc, lhlib):
    """5000 pairs: the tile-count scan carries its running total across five
    1024-pair chunks."""
    A, B, buf, vals_of = _batch(lhlib, 4, 5000, span_range=(16, 200), tiny=True)
    _check(ctx, orc, lhlib, A, B, vals_of, 5000)


def test_noalloc_at_its_limit(ctx, orc, lhlib):
    A, B, buf, vals_of = _batch(lhlib, 5, LIMIT, span_range=(16, 300), tiny=True)
    _check(ctx, orc, lhlib, A, B, vals_of, LIMIT)


def test_noalloc_leaves_the_pool_untouched(ctx, orc, lhlib):
    """No byte of the context's pool is handed out while the call runs: the
    pool's high-water mark, restarted before the call, stays at its current
    use."""
    import torch
    A, B, buf, vals_of = _batch(lhlib, 6, 200)
    got = torch.zeros(200, dtype=torch.int64, device="cuda")
    ctx.sync()
    now0, _ = ctx.pool_usage(reset_high=True)
    ctx.intersect_count_batch_noalloc(A, B, got)
    ctx.sync()
    now1, high = ctx.pool_usage()
    assert now1 == now0 and high == now0
    assert np.array_equal(got.cpu().numpy(), _oracle_counts(orc, vals_of))


def test_noalloc_rejects_batches_above_its_limit(ctx, lhlib):
    import torch
    lh = lhlib
    A, B, buf, vals_of = _batch(lh, 3, 2)
    counts = torch.full((2,), 7, dtype=torch.int64, device="cuda")
    with pytest.raises(lh.LHError) as e:
        ctx.intersect_count_batch_noalloc(A, B, counts, npairs=LIMIT + 1)
    assert e.value.status == lh.EINVAL and str(LIMIT) in str(e.value)
    assert counts.tolist() == [7, 7]
