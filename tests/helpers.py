"""Test-side helpers: move seeded inputs to the device and build the query
structs the C ABI takes.  No join arithmetic lives here."""
import numpy as np


def dev_u32(a):
    from paper_1708_07859_b300 import lh
    return lh.to_device_u32(a)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bitset_of(sorted_vals):
    """Pack a sorted set in the library's bitset format (base = min rounded
    down to 128, word count a multiple of 4): the layout, not the method."""
    v = np.asarray(sorted_vals, dtype=np.uint64)
    base = int(v[0]) & ~127 if v.size else 0
    nw = ((int(v[-1]) - base) >> 5) + 1 if v.size else 4
    nw = (nw + 3) & ~3
    words = np.zeros(nw, dtype=np.uint32)
    d = v - base
    np.bitwise_or.at(words, (d >> 5).astype(np.int64), (np.uint32(1) << (d & 31).astype(np.uint32)))
    return base, words


def graph_counts(ctx, src, dst, shape, orders, layouts=((32, 32),)):
    """COUNT of a graph pattern on the GPU under every (order, layout)."""
    from paper_1708_07859_b300 import lh
    s, d = dev_u32(src), dev_u32(dst)
    g = lh.GraphJoin(ctx, s, d, shape)
    out = {}
    try:
        for lay in layouts:
            for o in orders:
                plan = lh.make_plan(list(o), bs_ratio=lay[0])
                out[(tuple(o), tuple(lay))] = g.run(plan, layout=lay)[0]
    finally:
        g.free()
    return out
