"""Sparse LA as join-aggregates on the GPU vs the fp64 oracle:
SpMV y = A x (x completely dense) and SpGEMM C = A B in order [i, j, k];
componentwise |c - c64| <= 1e-6 * sum |a b|, exact sparsity pattern."""
import numpy as np
import pytest

from helpers import dev, dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu
TOL = 1e-6


def build(ctx, lh, coo):
    r, c, v = coo
    return lh.matrix_trie(ctx, dev_u32(r), dev_u32(c), dev(v))


def spmv(ctx, lh, coo, nrows, x):
    t = build(ctx, lh, coo)
    xd = dev(x)
    q = lh.spmv_query(nrows, xd, coo[0].size)
    r = ctx.join_aggregate(q, lh.make_plan([0, 1]), [t])
    v = r.wait()
    assert v.exec == lh.EXEC_SPMV
    y = r.y()
    r.free(); t.free()
    return y


@pytest.mark.parametrize("shape", [(300, 200, 7), (1000, 5000, 1), (64, 64, 64)])
def test_spmv_small(ctx, orc, lhlib, shape):
    n, m, k = shape
    coo = gen.uniform_coo(n, m, k, 31)
    x = gen.dense_vector(m, 32)
    y = spmv(ctx, lhlib, coo, n, x)
    w, wa = orc.spmv(*coo, n, x)
    assert np.all(np.abs(y - w) <= TOL * wa + 1e-30)


def test_spmv_identity_exact(ctx, lhlib):
    n = 5000
    x = gen.dense_vector(n, 3)
    y = spmv(ctx, lhlib, (np.arange(n), np.arange(n), np.ones(n, np.float32)), n, x)
    assert np.array_equal(y, x)


def test_spmv_full_size(ctx, orc, lhlib):
    n = 1 << 20
    coo = gen.zipf_coo(n, n)
    x = gen.dense_vector(n, gen.SEED_BASE + 20)
    y = spmv(ctx, lhlib, coo, n, x)
    w, wa = orc.spmv(*coo, n, x)
    assert np.all(np.abs(y - w) <= TOL * wa + 1e-30)


def spgemm(ctx, lh, A, B, group_impl=0):
    ta, tb = build(ctx, lh, A), build(ctx, lh, B)
    q = lh.spgemm_query(A[0].size, B[0].size, group_impl)
    r = ctx.join_aggregate(q, lh.make_plan([0, 1, 2]), [ta, tb])
    v = r.wait()
    assert v.exec == lh.EXEC_SPGEMM
    out = r.csr()
    r.free(); ta.free(); tb.free()
    return out


def check_rows(orc, A, nA, B, nB, ncols, rows_ids, off, cols, vals, sel_idx):
    sel = rows_ids[sel_idx]
    woff, wcol, wval, wabs = orc.spgemm_rows(A, nA, B, nB, ncols, sel)
    for s, p in enumerate(sel_idx):
        g0, g1 = int(off[p]), int(off[p + 1])
        w0, w1 = int(woff[s]), int(woff[s + 1])
        assert np.array_equal(cols[g0:g1], wcol[w0:w1]), int(sel[s])
        assert np.all(np.abs(vals[g0:g1] - wval[w0:w1]) <= TOL * wabs[w0:w1] + 1e-30)


@pytest.mark.parametrize("shape", [(200, 150, 180, 5, 4), (100, 3000, 80, 40, 30), (50, 50, 50, 50, 50)])
def test_spgemm_small(ctx, orc, lhlib, shape):
    nA, nB, nC, ka, kb = shape
    A = gen.uniform_coo(nA, nB, ka, 41)
    B = gen.uniform_coo(nB, nC, kb, 42)
    rows, off, cols, vals = spgemm(ctx, lhlib, A, B)
    assert np.array_equal(rows, np.unique(A[0]))
    check_rows(orc, A, nA, B, nB, nC, rows, off, cols, vals, np.arange(rows.size))


def test_spgemm_mixed_row_kinds(ctx, orc, lhlib):
    """Sort rows (uniform and ragged B rows), hash rows (more than 32 A
    entries, or more than 256 products), rows whose products are all missing
    and empty A rows, interleaved by row id: the rows are written in row order
    whatever kernel summed them."""
    nB, nC = 400, 300
    parts = []
    for i, k in enumerate((3, 40, 12, 1, 33, 2)):
        r, c, v = gen.uniform_coo(120, nB, k, 50 + i)
        parts.append((r * 7 + i, c, v))          # row ids 7r + i; 7r + 6 stay empty
    A = tuple(np.concatenate(x) for x in zip(*parts))
    r16, c16, v16 = gen.uniform_coo(200, nC, 16, 60)   # B rows 0..199: 16 entries
    r24, c24, v24 = gen.uniform_coo(120, nC, 24, 61)   # B rows 280..399: 24 entries
    B = (np.concatenate([r16, r24 + 280]).astype(np.uint32), np.concatenate([c16, c24]),
         np.concatenate([v16, v24]))                    # B rows 200..279 missing
    nA = 7 * 120
    rows, off, cols, vals = spgemm(ctx, lhlib, A, B)
    assert np.array_equal(rows, np.unique(A[0]))
    check_rows(orc, A, nA, B, nB, nC, rows, off, cols, vals, np.arange(rows.size))
    assert np.all(np.diff(off.astype(np.int64)) >= 0)


def test_spgemm_identity_and_permutation_exact(ctx, lhlib):
    A = gen.uniform_coo(300, 200, 9, 43)
    I = (np.arange(200), np.arange(200), np.ones(200, np.float32))
    rows, off, cols, vals = spgemm(ctx, lhlib, A, I)
    for p, i in enumerate(rows):
        m = A[0] == i
        o = np.argsort(A[1][m])
        assert np.array_equal(cols[off[p]:off[p + 1]], A[1][m][o])
        assert np.array_equal(vals[off[p]:off[p + 1]], A[2][m][o])


def test_spgemm_full_size_every_row(ctx, orc, lhlib):
    """Every row of C = A B at 2^20 x 2^20 (16 Zipf(1.1) columns per row):
    the CSR pattern (row offsets and columns) equals the oracle's exactly,
    so nnz(C) does too, and every value is within 1e-6 * sum |a b|."""
    n = 1 << 20
    A = gen.zipf_coo(n, n)
    B = gen.zipf_coo(n, n, seed=gen.SEED_BASE + 12)
    rows, off, cols, vals = spgemm(ctx, lhlib, A, B)
    assert np.array_equal(rows, np.arange(n, dtype=rows.dtype))
    woff, wcol, wval, wabs = orc.spgemm_rows(A, n, B, n, n, np.arange(n, dtype=np.uint32))
    assert int(off[-1]) == int(woff[-1]) == cols.size
    assert np.array_equal(off.astype(np.uint64), woff)
    assert np.array_equal(cols, wcol)
    err = np.abs(vals.astype(np.float64) - wval)
    bad = err > TOL * wabs + 1e-30
    assert not bad.any(), (int(bad.sum()), float(np.max(err / np.maximum(wabs, 1e-30))))


@pytest.mark.parametrize("impl", ["auto", "dense", "sort_hash"])
def test_spgemm_group_by_key_implementations(ctx, orc, lhlib, impl):
    """Section 5 GROUP BY key: banded matrices whose products fill narrow
    column spans (dense rows: bitset + dense array under the density rule),
    next to rows too wide for the dense array and sparse Zipf rows; every
    implementation choice gives the oracle's C."""
    lh = lhlib
    gi = {"auto": lh.GROUP_AUTO, "dense": lh.GROUP_DENSE, "sort_hash": lh.GROUP_PRIVATE}[impl]
    n = 3000
    Ab = gen.banded_coo(n, n, 40, 200, 71)          # 40 entries per row: not a sort row
    Bb = gen.banded_coo(n, n, 24, 300, 72)
    Az = gen.uniform_coo(500, n, 6, 73)              # sparse rows over the whole range
    A = (np.concatenate([Ab[0], Az[0] + n]), np.concatenate([Ab[1], Az[1]]), np.concatenate([Ab[2], Az[2]]))
    nA = n + 500
    rows, off, cols, vals = spgemm(ctx, lh, A, Bb, gi)
    assert np.array_equal(rows, np.unique(A[0]))
    woff, wcol, wval, wabs = orc.spgemm_rows(A, nA, Bb, n, n, rows)
    assert np.array_equal(off.astype(np.uint64), woff) and np.array_equal(cols, wcol)
    assert np.all(np.abs(vals - wval) <= TOL * wabs + 1e-30)


def test_spgemm_dense_rows_wider_than_the_array(ctx, orc, lhlib):
    """Forcing the dense accumulator: rows whose span exceeds it fall back to
    the hash path, exactly."""
    lh = lhlib
    n = 20000
    A = gen.banded_coo(n, n, 20, 6000, 74)
    B = gen.banded_coo(n, n, 10, 3000, 75)
    rows, off, cols, vals = spgemm(ctx, lh, A, B, lh.GROUP_DENSE)
    woff, wcol, wval, wabs = orc.spgemm_rows(A, n, B, n, n, rows)
    assert np.array_equal(off.astype(np.uint64), woff) and np.array_equal(cols, wcol)
    assert np.all(np.abs(vals - wval) <= TOL * wabs + 1e-30)
