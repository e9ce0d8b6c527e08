"""Trie build (Section 2.2) on the GPU vs the oracle's sorted-unique levels;
bitset words and ranks vs the set's own elements; filter relations
(Section 3.2) vs the plain predicate."""
import itertools

import numpy as np
import pytest

from helpers import dev, dev_u32
from paper_1708_07859_b300 import inputs as gen

pytestmark = pytest.mark.gpu


def check_bitsets(tr, lv_index, arrays, words, rank):
    """Every bitset set holds exactly its elements; rank = bits before the word."""
    lv = arrays[lv_index]
    if lv["n_bs"] == 0:
        return 0
    prev = arrays[lv_index - 1] if lv_index > 0 else None
    nsets = 1 if lv_index == 0 else prev["vals"].size
    checked = 0
    # arena-wide rank: bits of all earlier words (popcounts from the bytes)
    all_pc = np.unpackbits(np.ascontiguousarray(words).view(np.uint8)).reshape(-1, 32).sum(axis=1).astype(np.int64)
    prefix = np.concatenate([[0], np.cumsum(all_pc)[:-1]])
    for s in range(nsets):
        slot = lv["bs_slot"][s]
        if slot == 0xFFFFFFFF:
            continue
        lo, hi = (0, lv["vals"].size) if lv_index == 0 else (int(prev["offs"][s]), int(prev["offs"][s + 1]))
        elems = lv["vals"][lo:hi].astype(np.int64)
        w0, base, nw, rbase = (int(x) for x in lv["bs_meta"][slot])
        assert base == (int(elems[0]) & ~127) and nw % 4 == 0 and w0 % 4 == 0
        ws = words[w0:w0 + nw]
        bits = np.unpackbits(ws.view(np.uint8), bitorder="little").astype(bool)
        assert np.array_equal(np.flatnonzero(bits) + base, elems)
        # rank base = rank of the set's first word
        assert rbase == prefix[w0]
        assert np.array_equal(rank[w0:w0 + nw].astype(np.int64), prefix[w0:w0 + nw])
        checked += 1
    return checked


@pytest.mark.parametrize("seed", [0, 1])
def test_trie_levels_match_oracle(ctx, orc, seed):
    rng = np.random.default_rng(seed)
    n = 5000
    cols = [rng.integers(0, 50, n), rng.integers(0, 3000, n), rng.integers(0, 7, n)]
    dcols = [dev_u32(c) for c in cols]
    for order in itertools.permutations(range(3)):
        tr = ctx.build_trie(dcols, key_order=list(order))
        want = orc.trie_levels(cols, order)
        arrays = [tr.level_arrays(l) for l in range(3)]
        for l in range(3):
            assert np.array_equal(arrays[l]["vals"], want[l][0]), (order, l)
            if l > 0:
                assert np.array_equal(arrays[l - 1]["offs"].astype(np.uint64), want[l][1]), (order, l)
        words, rank = tr.words()
        for l in range(3):
            check_bitsets(tr, l, arrays, words, rank)
        st = tr.stats()
        assert st.nrows_in == n and list(st.key_order)[:3] == list(order)
        tr.free()


def test_layout_policy_decides_bitsets(ctx):
    # level 0 dense (all of 0..4095), level 1 sparse children
    src, dst = gen.triangle_workload()
    s, d = dev_u32(src), dev_u32(dst)
    t_default = ctx.build_trie([s, d])
    st = t_default.stats()
    assert st.level_bs_sets[0] == 1 and st.level_bs_sets[1] == 0
    words, rank = t_default.words()
    arrays = [t_default.level_arrays(l) for l in range(2)]
    assert check_bitsets(t_default, 0, arrays, words, rank) == 1
    t_uint = ctx.build_trie([s, d], layout=(0, 0))
    assert t_uint.stats().level_bs_sets[0] == 0 and t_uint.stats().bitset_words == 0
    t_all = ctx.build_trie([s, d], layout=(4096, 1))    # every set a bitset
    st = t_all.stats()
    assert st.level_bs_sets[1] == st.level_sets[1]
    arrays = [t_all.level_arrays(l) for l in range(2)]
    words, rank = t_all.words()
    assert check_bitsets(t_all, 1, arrays, words, rank) == st.level_sets[1]
    for t in (t_default, t_uint, t_all):
        t.free()


def test_sum_merge_of_duplicate_tuples(ctx):
    rng = np.random.default_rng(4)
    n = 20000
    a = rng.integers(0, 40, n)
    b = rng.integers(0, 40, n)
    v = rng.uniform(-1, 1, n).astype(np.float32)
    from paper_1708_07859_b300 import lh
    tr = ctx.build_trie([dev_u32(a), dev_u32(b)], annos=[(dev(v), lh.T_F32)], merge=lh.MERGE_SUM)
    got = tr.anno_array(0)
    key = a * 40 + b
    uk, inv = np.unique(key, return_inverse=True)
    want = np.zeros(uk.size)
    np.add.at(want, inv, v.astype(np.float64))
    assert got.size == uk.size
    cnt = np.bincount(inv)
    assert np.all(np.abs(got - want) <= 1e-6 * cnt * np.maximum(1.0, np.abs(want)))
    tr.free()


@pytest.mark.parametrize("dups", [True, False])
def test_annotation_merge_paths(ctx, dups):
    """FIRST keeps the first input row of each distinct tuple, SUM adds the
    rows; one 4-byte column (sorted along with the keys) and the other
    column shapes (gathered through row ids) give the same leaf order."""
    from paper_1708_07859_b300 import lh
    rng = np.random.default_rng(9)
    n = 9000
    if dups:
        a, b = rng.integers(0, 30, n), rng.integers(0, 60, n)
    else:
        key = rng.permutation(70 * 200)[:n]
        a, b = key // 200, key % 200
    key = a.astype(np.int64) * 1000 + b
    uk, first, inv = np.unique(key, return_index=True, return_inverse=True)
    u32 = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    f32 = rng.uniform(-1, 1, n).astype(np.float32)
    f64 = rng.uniform(-1, 1, n)
    i8 = rng.integers(-100, 100, n).astype(np.int8)
    da, db = dev_u32(a), dev_u32(b)
    cases = [([(u32, lh.T_U32)], lh.MERGE_FIRST), ([(f32, lh.T_F32)], lh.MERGE_FIRST),
             ([(i8, lh.T_I8)], lh.MERGE_FIRST), ([(f32, lh.T_F32), (u32, lh.T_U32)], lh.MERGE_FIRST),
             ([(f64, lh.T_F64)], lh.MERGE_SUM), ([(f32, lh.T_F32)], lh.MERGE_SUM)]
    for annos, merge in cases:
        tr = ctx.build_trie([da, db], annos=[(dev(x), ty) for x, ty in annos], merge=merge)
        assert tr.stats().level_n[1] == uk.size
        for c, (x, ty) in enumerate(annos):
            got = tr.anno_array(c)
            if merge == lh.MERGE_FIRST:
                assert np.array_equal(got, x[first]), (ty, merge)
            else:
                want = np.zeros(uk.size)
                np.add.at(want, inv, x.astype(np.float64))
                cnt = np.bincount(inv)
                tol = (1e-6 if ty == lh.T_F32 else 1e-13) * cnt * np.maximum(1.0, np.abs(want))
                assert np.all(np.abs(got - want) <= tol), (ty, merge)
        tr.free()


def test_price_discount_expression_annotation(ctx):
    data = gen.star_schema(4000, dims=(50, 40, 30, 5), seed=11)
    from paper_1708_07859_b300 import lh
    keys = [dev_u32(k) for k in data["k"]]
    tr = ctx.build_trie(keys, annos=[(dev(data["price"]), lh.T_F64), (dev(data["disc"]), lh.T_I8)],
                        merge=lh.MERGE_PRICE_DISCOUNT)
    hi, lo = tr.anno_array(0).astype(np.float64), tr.anno_array(1).astype(np.float64)
    k = data["k"]
    packed = ((k[0].astype(np.uint64) * 40 + k[1]) * 30 + k[2]) * 5 + k[3]
    uk, inv = np.unique(packed, return_inverse=True)
    want = np.zeros(uk.size)
    np.add.at(want, inv, data["price"] * (1.0 - data["disc"] / 100.0))
    # fp32 price rounding dominates: each term is within 2^-23 relative
    assert np.all(np.abs(hi + lo - want) <= 2.5e-7 * want)
    tr.free()


def test_filter_trie_matches_predicate(ctx, orc):
    rng = np.random.default_rng(2)
    col = rng.integers(0, 2557, 200_000).astype(np.int32)
    for lo, hi in [(0, 2556), (100, 150), (3000, 4000), (2000, 1000)]:
        tr = ctx.filter_trie(dev(col), lo, hi)
        got = tr.level_arrays(0)["vals"]
        assert np.array_equal(got, orc.filter_keys(col, lo, hi))
        tr.free()


def test_empty_relation(ctx):
    e = dev_u32(np.zeros(0, np.uint32))
    tr = ctx.build_trie([e, e])
    st = tr.stats()
    assert st.level_n[0] == 0 and st.level_n[1] == 0
    tr.free()


def test_declared_key_bounds(ctx, orc):
    """Key domains declared by the caller give the same trie as the maxima
    read from the columns; a value at or above its bound is refused."""
    from paper_1708_07859_b300 import lh
    rng = np.random.default_rng(12)
    n = 7000
    cols = [rng.integers(0, 300, n), rng.integers(0, 5000, n)]
    dcols = [dev_u32(c) for c in cols]
    want = orc.trie_levels(cols, (0, 1))
    for bounds in ((300, 5000), (1 << 12, 1 << 20)):
        tr = ctx.build_trie(dcols, key_bounds=bounds)
        arrays = [tr.level_arrays(l) for l in range(2)]
        assert np.array_equal(arrays[0]["vals"], want[0][0])
        assert np.array_equal(arrays[1]["vals"], want[1][0])
        assert np.array_equal(arrays[0]["offs"].astype(np.uint64), want[1][1])
        tr.free()
    with pytest.raises(lh.LHError) as e:
        ctx.build_trie(dcols, key_bounds=(300, 4000))
    assert e.value.status == lh.EINVAL
