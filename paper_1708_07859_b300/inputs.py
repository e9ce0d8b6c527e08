"""Seeded synthetic input generators shared by the oracle tests, the GPU tests
and the benchmark.

This module holds no join, intersection or aggregation arithmetic: it only
draws relations (edge lists, sparse matrices, star-schema tables, dense
blocks) from numpy ``PCG64`` streams, so that the CPU oracle and the CUDA path
read byte-identical inputs.  Every generator is a pure function of its
arguments and seed.

Workload shapes follow the evaluation of the paper (Section 6): graph
relations for worst-case-optimal joins, sparse matrices whose product is a
join-aggregate (Section 4.1.2 example), a star-schema BI join with filters and
GROUP BY (Sections 2.1, 3.1, 5), and dense blocks (Section 3.1, attribute
elimination).  Public datasets the paper used are not available; these
generators stand in for them.
"""
from __future__ import annotations

import math
import numpy as np

SEED_BASE = 1708078590


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


# --------------------------------------------------------------------------
# graphs (binary relations E(src, dst), oriented src < dst, distinct)
# --------------------------------------------------------------------------

def _canon_unique(u: np.ndarray, v: np.ndarray, n: int):
    """Drop self loops, orient min->max, return unique packed keys (sorted)."""
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.minimum(u, v).astype(np.uint64)
    b = np.maximum(u, v).astype(np.uint64)
    return np.unique(a * np.uint64(n) + b)


def gnm_edges(n: int, m: int, seed: int):
    """G(n, m): ``m`` distinct undirected pairs drawn uniformly without
    replacement from the C(n, 2) possible ones, oriented min->max, returned in
    a random order as two uint32 arrays."""
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds C(n,2)")
    rng = _rng(seed)
    keys = np.zeros(0, dtype=np.uint64)
    batch = max(1024, int(m * 1.3))
    while keys.size < m:
        u = rng.integers(0, n, size=batch, dtype=np.int64)
        v = rng.integers(0, n, size=batch, dtype=np.int64)
        keys = np.union1d(keys, _canon_unique(u, v, n))
    if keys.size > m:
        keys = rng.choice(keys, size=m, replace=False)
    rng.shuffle(keys)
    src = (keys // np.uint64(n)).astype(np.uint32)
    dst = (keys % np.uint64(n)).astype(np.uint32)
    return src, dst


def chung_lu_edges(n: int, m: int, beta: float, seed: int):
    """Chung-Lu power-law graph: endpoint v drawn with probability
    proportional to w_v = (v+1)^(-1/(beta-1)) (vertex 0 heaviest), self loops
    and repeats dropped, pairs taken in draw order until exactly ``m``
    distinct edges exist.  Oriented min->max (hubs have low ids, so their
    out-sets are the dense ones)."""
    rng = _rng(seed)
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -1.0 / (beta - 1.0))
    cdf = np.cumsum(w)
    total = cdf[-1]
    seen_keys = np.zeros(0, dtype=np.uint64)
    order_keys = []
    have = 0
    batch = max(4096, int(m * 1.5))
    while have < m:
        u = np.searchsorted(cdf, rng.random(batch) * total, side="right")
        v = np.searchsorted(cdf, rng.random(batch) * total, side="right")
        u = np.minimum(u, n - 1)
        v = np.minimum(v, n - 1)
        keep = u != v
        a = np.minimum(u[keep], v[keep]).astype(np.uint64)
        b = np.maximum(u[keep], v[keep]).astype(np.uint64)
        k = a * np.uint64(n) + b
        # first occurrence within this batch, in draw order
        _, first = np.unique(k, return_index=True)
        first.sort()
        k = k[first]
        k = k[~np.isin(k, seen_keys, assume_unique=True)]
        need = m - have
        k = k[:need]
        order_keys.append(k)
        have += k.size
        if have < m:
            # k holds distinct keys none of which was seen: the union is the
            # sorted concatenation
            seen_keys = np.sort(np.concatenate([seen_keys, k]))
    keys = np.concatenate(order_keys)
    src = (keys // np.uint64(n)).astype(np.uint32)
    dst = (keys % np.uint64(n)).astype(np.uint32)
    return src, dst


def complete_graph(n: int):
    a, b = np.triu_indices(n, k=1)
    return a.astype(np.uint32), b.astype(np.uint32)


def complete_bipartite(p: int, q: int):
    a = np.repeat(np.arange(p), q)
    b = np.tile(np.arange(p, p + q), p)
    return a.astype(np.uint32), b.astype(np.uint32)


def cycle_graph(n: int):
    a = np.arange(n)
    b = (a + 1) % n
    return np.minimum(a, b).astype(np.uint32), np.maximum(a, b).astype(np.uint32)


def wheel_graph(n: int):
    """Hub 0 joined to the n-cycle on vertices 1..n."""
    ring = np.arange(1, n + 1)
    nxt = np.where(ring == n, 1, ring + 1)
    a = np.concatenate([np.zeros(n, dtype=np.int64), np.minimum(ring, nxt)])
    b = np.concatenate([ring, np.maximum(ring, nxt)])
    return a.astype(np.uint32), b.astype(np.uint32)


def triangle_workload(seed_offset: int = 1, n: int = 4096, m: int = 32768):
    """Uniform random graph used for the 3-way triangle join: 4096 vertices,
    32768 distinct oriented edges."""
    return gnm_edges(n, m, SEED_BASE + seed_offset)


def batch_graph_sizes(count: int = 4096, seed_offset: int = 4):
    """Edge counts m_i = round(exp(U[ln 100, ln 1e5])) and vertex counts
    n_i = max(16, ceil(m_i / 8), smallest n with C(n, 2) >= m_i) for a batch
    of independent graphs."""
    rng = _rng(SEED_BASE + seed_offset)
    m = np.rint(np.exp(rng.uniform(math.log(100.0), math.log(1e5), size=count))).astype(np.int64)
    n = np.maximum(16, np.ceil(m / 8.0)).astype(np.int64)
    # at least enough vertices for m distinct pairs: C(n, 2) >= m
    n_min = np.ceil((1.0 + np.sqrt(1.0 + 8.0 * m)) / 2.0).astype(np.int64)
    return np.maximum(n, n_min), m


def batch_graph(i: int, n: int, m: int, seed_offset: int = 4):
    return gnm_edges(int(n), int(m), SEED_BASE + seed_offset + 1 + int(i))


def _batch_graph_args(args):
    return batch_graph(*args)


def batch_graphs(count: int = 4096, seed_offset: int = 4, workers: int = 0):
    """The ``count`` graphs of a batch (graph i is ``batch_graph(i, n_i,
    m_i)``), drawn in parallel by a pool of fresh (spawned) worker processes
    when ``workers`` != 1; every graph has its own seed, so the result does
    not depend on the pool.  workers 0 = one per host core."""
    ns, ms = batch_graph_sizes(count, seed_offset)
    args = [(i, int(ns[i]), int(ms[i]), seed_offset) for i in range(count)]
    import os
    w = workers or (os.cpu_count() or 1)
    if w <= 1 or count < 64:
        return [batch_graph(*a) for a in args]
    import concurrent.futures as cf
    import multiprocessing as mp
    # fresh interpreters (a forked CUDA process would hang); a worker that
    # dies raises BrokenProcessPool here instead of leaving the map waiting
    with cf.ProcessPoolExecutor(min(w, 32), mp_context=mp.get_context("spawn")) as pool:
        return list(pool.map(_batch_graph_args, args, chunksize=32, timeout=1800))


HUB_GRAPH = (1 << 20, 1 << 24, 2.1)   # n, m, degree exponent of the power-law batch graph


def hub_graph(seed_offset: int = 4):
    """The power-law graph that joins the uneven batch: Chung-Lu with 2^24
    distinct edges over 2^20 vertices, degree exponent 2.1 (hub out-sets are
    dense enough for the bitset layout)."""
    n, m, beta = HUB_GRAPH
    return chung_lu_edges(n, m, beta, SEED_BASE + seed_offset)


# --------------------------------------------------------------------------
# sparse matrices (relations A(i, j) with an fp32 annotation)
# --------------------------------------------------------------------------

def zipf_coo(nrows: int, ncols: int, per_row: int = 16, s: float = 1.1,
             seed: int = SEED_BASE + 2, chunk: int = 1 << 16):
    """Sparse matrix with exactly ``per_row`` distinct columns per row.

    Column index = rank - 1 with rank drawn from Zipf(s) truncated to
    [1, ncols] (P(r) proportional to r^-s, hot columns are low ids); each row
    redraws until it has ``per_row`` distinct columns (first occurrences in
    draw order).  Values fp32 U[-1, 1].  Returns COO (rows, cols, vals) in row
    order, columns in draw order within a row.
    """
    rng = _rng(seed)
    cdf = np.cumsum(np.power(np.arange(1, ncols + 1, dtype=np.float64), -s))
    total = cdf[-1]
    rows_out, cols_out = [], []
    draws = per_row * 3
    for r0 in range(0, nrows, chunk):
        r1 = min(nrows, r0 + chunk)
        nr = r1 - r0
        out = np.empty((nr, per_row), dtype=np.int64)
        pending = np.arange(nr)
        while pending.size:
            cand = np.searchsorted(cdf, rng.random((pending.size, draws)) * total, side="right")
            cand = np.minimum(cand, ncols - 1)
            order = np.argsort(cand, axis=1, kind="stable")
            srt = np.take_along_axis(cand, order, axis=1)
            dup_sorted = np.zeros_like(srt, dtype=bool)
            dup_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
            first = np.ones_like(cand, dtype=bool)
            np.put_along_axis(first, order, ~dup_sorted, axis=1)
            rank = np.cumsum(first, axis=1)
            ok = rank[:, -1] >= per_row
            take = first & (rank <= per_row)
            done = pending[ok]
            out[done] = cand[ok][take[ok]].reshape(-1, per_row)
            pending = pending[~ok]
        rows_out.append(np.repeat(np.arange(r0, r1, dtype=np.int64), per_row))
        cols_out.append(out.reshape(-1))
    rows = np.concatenate(rows_out).astype(np.uint32)
    cols = np.concatenate(cols_out).astype(np.uint32)
    vals = rng.uniform(-1.0, 1.0, size=rows.size).astype(np.float32)
    return rows, cols, vals


def banded_coo(nrows: int, ncols: int, per_row: int, width: int, seed: int):
    """Sparse matrix whose row i holds ``per_row`` distinct columns drawn
    uniformly from the band [i*ncols/nrows, i*ncols/nrows + width) (clipped
    to the matrix); values fp32 U[-1, 1].  Products of banded matrices fill
    narrow column ranges densely (the structured matrices of the paper's
    sparse LA experiments)."""
    rng = _rng(seed)
    width = min(width, ncols)
    starts = np.minimum((np.arange(nrows, dtype=np.int64) * ncols) // nrows, ncols - width)
    # per_row distinct offsets in [0, width): the first per_row of a random ordering
    offs = np.argsort(rng.random((nrows, width)), axis=1)[:, :per_row]
    cols = (starts[:, None] + offs).reshape(-1)
    rows = np.repeat(np.arange(nrows, dtype=np.int64), per_row)
    vals = rng.uniform(-1.0, 1.0, size=rows.size).astype(np.float32)
    return rows.astype(np.uint32), cols.astype(np.uint32), vals


def uniform_coo(nrows: int, ncols: int, per_row: int, seed: int):
    """Small sparse matrix with ``per_row`` distinct uniform columns per row."""
    rng = _rng(seed)
    cols = np.stack([rng.choice(ncols, size=per_row, replace=False) for _ in range(nrows)])
    rows = np.repeat(np.arange(nrows), per_row)
    vals = rng.uniform(-1.0, 1.0, size=rows.size).astype(np.float32)
    return rows.astype(np.uint32), cols.reshape(-1).astype(np.uint32), vals


def dense_vector(n: int, seed: int):
    return _rng(seed).uniform(-1.0, 1.0, size=n).astype(np.float32)


def dense_matrix(rows: int, cols: int, seed: int):
    return _rng(seed).uniform(-1.0, 1.0, size=(rows, cols)).astype(np.float32)


# --------------------------------------------------------------------------
# star schema (fact table with foreign keys into four dimensions)
# --------------------------------------------------------------------------

DIM_SIZES = (1_500_000, 200_000, 10_000, 25)
DATE_DAYS = 2557


def star_schema(n_fact: int = 60_000_000, dims=DIM_SIZES, seed: int = SEED_BASE + 3):
    """Fact(k1..k4, price, discount) with uniform int foreign keys into four
    dimensions and dimension attribute columns.

    price fp64 U[900, 105000]; discount in hundredths U{0..10} (int8).
    D1: d1_date U[0, 2557), d1_seg U[0, 5); D2: d2_cat U[0, 40);
    D3: d3_grp U[0, 100); D4: d4_region U[0, 5).
    """
    rng = _rng(seed)
    keys = [rng.integers(0, d, size=n_fact, dtype=np.int64).astype(np.uint32) for d in dims]
    price = rng.uniform(900.0, 105000.0, size=n_fact)
    disc = rng.integers(0, 11, size=n_fact, dtype=np.int64).astype(np.int8)
    d1_date = rng.integers(0, DATE_DAYS, size=dims[0], dtype=np.int64).astype(np.int32)
    d1_seg = rng.integers(0, 5, size=dims[0], dtype=np.int64).astype(np.int32)
    d2_cat = rng.integers(0, 40, size=dims[1], dtype=np.int64).astype(np.int32)
    d3_grp = rng.integers(0, 100, size=dims[2], dtype=np.int64).astype(np.int32)
    d4_region = rng.integers(0, 5, size=dims[3], dtype=np.int64).astype(np.int32)
    return {
        "k": keys, "price": price, "disc": disc,
        "d1_date": d1_date, "d1_seg": d1_seg, "d2_cat": d2_cat,
        "d3_grp": d3_grp, "d4_region": d4_region,
    }


BI_SIZES = {"fact": 60_000_000, "orders": 15_000_000, "customer": 1_500_000, "supplier": 100_000,
            "nation": 25, "region": 5}


def bi_schema(sizes=None, seed: int = SEED_BASE + 6):
    """A six-relation BI schema shaped like the paper's two-node example
    query (Section 3.1: a fact relation over (order, supplier), orders over
    (order, customer), customer and supplier over a shared nation key, nation
    over a region key, region): every relation's first key is its row id;
    foreign keys uniform; fact price fp64 U[900, 105000] and discount
    U{0..10} hundredths; orders carry a date U[0, 2557); region and nation a
    name code (their row id).  Relation and column names are this
    generator's own."""
    z = dict(BI_SIZES)
    z.update(sizes or {})
    rng = _rng(seed)
    u32 = lambda hi, n: rng.integers(0, hi, size=n, dtype=np.int64).astype(np.uint32)
    nf = z["fact"]
    # distinct (order, supplier) pairs, first occurrences in draw order: a
    # fact row is identified by its key tuple
    no, ns = z["orders"], z["supplier"]
    if nf > no * ns:
        raise ValueError("more fact rows than (order, supplier) pairs")
    keys = np.zeros(0, dtype=np.uint64)
    while keys.size < nf:
        draw = rng.integers(0, no, size=nf + 64, dtype=np.int64).astype(np.uint64) * np.uint64(ns) + \
            rng.integers(0, ns, size=nf + 64, dtype=np.int64).astype(np.uint64)
        allk = np.concatenate([keys, draw])
        _, first = np.unique(allk, return_index=True)
        first.sort()
        keys = allk[first][:nf]
    return {
        "sizes": z,
        "fact_order": (keys // np.uint64(ns)).astype(np.uint32), "fact_supp": (keys % np.uint64(ns)).astype(np.uint32),
        "price": rng.uniform(900.0, 105000.0, size=nf),
        "disc": rng.integers(0, 11, size=nf, dtype=np.int64).astype(np.int8),
        "order_cust": u32(z["customer"], z["orders"]),
        "order_date": rng.integers(0, DATE_DAYS, size=z["orders"], dtype=np.int64).astype(np.int32),
        "cust_nation": u32(z["nation"], z["customer"]),
        "supp_nation": u32(z["nation"], z["supplier"]),
        "nation_region": u32(z["region"], z["nation"]),
        "nation_name": np.arange(z["nation"], dtype=np.int32),
        "region_name": np.arange(z["region"], dtype=np.int32),
    }


def date_range_for_selectivity(sel: float):
    """Inclusive [lo, hi] day range on d1_date keeping about ``sel`` of days."""
    width = max(1, int(round(sel * DATE_DAYS)))
    lo = (DATE_DAYS - width) // 2
    return lo, lo + width - 1


# --------------------------------------------------------------------------
# sorted sets for the intersection micro-benchmark (Figure 4a shapes)
# --------------------------------------------------------------------------

def sorted_set(card: int, span: int, seed: int):
    """``card`` distinct uint32 values drawn uniformly from [0, span), sorted."""
    rng = _rng(seed)
    if card * 4 >= span:
        v = np.flatnonzero(rng.random(span) < (card / span))
    else:
        v = np.unique(rng.integers(0, span, size=int(card * 1.1) + 16))
        while v.size < card:
            v = np.union1d(v, rng.integers(0, span, size=card))
        v = np.sort(rng.choice(v, size=card, replace=False))
    return v.astype(np.uint32)


def gap_set(card: int, mean_gap: float, seed: int, start: int = 0):
    """``card`` distinct sorted uint32 values whose consecutive gaps are
    Geometric(1/mean_gap): a uniform random set of density ~1/mean_gap.
    Cheap enough to draw hundreds of million-element sets."""
    rng = _rng(seed)
    gaps = rng.geometric(1.0 / mean_gap, size=card)
    v = start + np.cumsum(gaps) - gaps[0]
    if v.size and v[-1] >= (1 << 32):
        raise ValueError("set exceeds the uint32 domain")
    return v.astype(np.uint32)
