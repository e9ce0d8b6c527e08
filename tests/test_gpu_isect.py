"""Count-only set intersections (Section 4.1.1 layouts, Figure 4a shapes) on
the GPU vs the oracle's plain merge; every layout pairing, skewed sizes,
empty sets and ragged tails."""
import numpy as np
import pytest

from helpers import bitset_of, dev, dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu


def run_pairs(ctx, lh, pairs):
    """pairs: list of ((layout, vals), (layout, vals)); returns GPU counts."""
    import torch
    keep = []
    descs = {0: [], 1: []}
    for pa, pb in pairs:
        for side, (layout, vals) in zip((0, 1), (pa, pb)):
            if layout == 0:
                t = dev_u32(vals) if len(vals) else dev_u32(np.zeros(1, np.uint32))
                keep.append(t)
                descs[side].append((0, 0, len(vals), t.data_ptr()))
            else:
                base, words = bitset_of(vals)
                t = dev_u32(words)
                keep.append(t)
                descs[side].append((1, base, words.size, t.data_ptr()))
    A = torch.frombuffer(bytearray(lh.pack_sets(descs[0])), dtype=torch.uint8).cuda()
    B = torch.frombuffer(bytearray(lh.pack_sets(descs[1])), dtype=torch.uint8).cuda()
    counts = torch.zeros(len(pairs), dtype=torch.int64, device="cuda")
    ctx.intersect_count_batch(A, B, counts)
    torch.cuda.synchronize()
    return counts.cpu().numpy().astype(np.uint64)


def test_all_layout_pairs_and_edge_cases(ctx, orc, lhlib):
    S = lambda c, span, seed: gen.sorted_set(c, span, seed)
    raw = [
        (S(1000, 4000, 1), S(1000, 4000, 2)),            # balanced, dense-ish
        (S(4096 * 3 + 17, 200000, 3), S(4096 * 2 + 5, 200000, 4)),  # ragged tiles
        (S(100, 10**6, 5), S(100000, 10**6, 6)),         # skew > 32: probe path
        (S(100000, 10**6, 7), S(100, 10**6, 8)),         # skew, swapped
        (np.zeros(0, np.uint32), S(50, 100, 9)),         # empty side
        (np.array([7], np.uint32), np.array([7], np.uint32)),
        (np.array([7], np.uint32), np.array([8], np.uint32)),
        (np.arange(0, 5000, 2, dtype=np.uint32), np.arange(1, 5000, 2, dtype=np.uint32)),  # disjoint interleaved
        (np.arange(10**5, dtype=np.uint32), np.arange(10**5, dtype=np.uint32)),             # identical
        (S(30000, 60000, 10), S(30000, 60000, 11)),
        (S(5000, 10**6, 12) + 300000, S(8000, 400000, 13)),  # partial overlap of ranges
    ]
    pairs = []
    for a, b in raw:
        for la, lb in [(0, 0), (0, 1), (1, 0), (1, 1)]:
            if (la == 1 and a.size == 0) or (lb == 1 and b.size == 0):
                continue
            pairs.append(((la, a), (lb, b)))
    got = run_pairs(ctx, lhlib, pairs)
    want = np.array([orc.intersect_count(a, b) for (_, a), (_, b) in pairs], dtype=np.uint64)
    assert np.array_equal(got, want)


def test_figure4a_shapes_at_1e6(ctx, orc, lhlib):
    # equal-cardinality sets (card 1e6, density 1/2) in all three layouts, and
    # sparse uint sets (span 32 x card)
    pairs = []
    for p in range(4):
        a = gen.sorted_set(10**6, 2 * 10**6, 100 + p)
        b = gen.sorted_set(10**6, 2 * 10**6, 200 + p)
        pairs += [((0, a), (0, b)), ((0, a), (1, b)), ((1, a), (1, b))]
        a = gen.sorted_set(10**6, 32 * 10**6, 300 + p)
        b = gen.sorted_set(10**6, 32 * 10**6, 400 + p)
        pairs.append(((0, a), (0, b)))
    got = run_pairs(ctx, lhlib, pairs)
    want = np.array([orc.intersect_count(a, b) for (_, a), (_, b) in pairs], dtype=np.uint64)
    assert np.array_equal(got, want)
