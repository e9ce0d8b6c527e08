// Trie construction (Section 2.2): key tuples packed in attribute order,
// radix-sorted, deduplicated with annotation merge, emitted as CSR levels;
// each set then gets the uint or bitset layout; annotations are gathered into
// leaf order (Section 3.1: each annotation in its own buffer).  Also the
// filter relation of a pushed-down selection (Section 3.2).
#include "lh_internal.cuh"

namespace {

__global__ void k_col_max(const uint32_t *col, uint64_t n, uint32_t *out) {
    uint32_t m = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, col[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(LH_FULL, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

struct PackArgs {
    const uint32_t *col[LH_MAX_LEVELS];
    uint32_t shift[LH_MAX_LEVELS];
    uint32_t nlev;
};

__global__ void k_pack(PackArgs a, uint64_t n, uint64_t *key, uint32_t *rid) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = 0;
        for (uint32_t l = 0; l < a.nlev; ++l) k |= (uint64_t)a.col[l][i] << a.shift[l];
        key[i] = k;
        rid[i] = (uint32_t)i;
    }
}

// head flags of distinct keys
__global__ void k_heads(const uint64_t *key, uint64_t n, uint32_t *flag) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || key[i] != key[i - 1]) ? 1u : 0u;
}

// compact distinct keys; runstart[u] = first sorted row of distinct tuple u
__global__ void k_compact_unique(const uint64_t *key, const uint32_t *flag, const uint64_t *pos,
                                 uint64_t n, uint64_t *ukey, uint64_t *runstart) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (flag[i]) {
            ukey[pos[i]] = key[i];
            runstart[pos[i]] = i;
        }
}

// per-level prefix-boundary flags over distinct keys
__global__ void k_level_flags(const uint64_t *ukey, uint64_t nu, uint32_t pshift, uint32_t *flag) {
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu;
         u += (uint64_t)gridDim.x * blockDim.x) {
        bool h = (u == 0);
        if (!h) {
            uint64_t a = pshift >= 64 ? 0 : (ukey[u] >> pshift);
            uint64_t b = pshift >= 64 ? 0 : (ukey[u - 1] >> pshift);
            h = a != b;
        }
        flag[u] = h ? 1u : 0u;
    }
}

__global__ void k_level_emit(const uint64_t *ukey, uint64_t nu, const uint32_t *flag,
                             const uint32_t *pos, uint32_t vshift, uint64_t vmask, uint32_t *vals,
                             const uint32_t *pflag, const uint32_t *ppos, uint32_t *poffs) {
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu;
         u += (uint64_t)gridDim.x * blockDim.x) {
        if (!flag[u]) continue;
        uint32_t p = pos[u];
        vals[p] = (uint32_t)((ukey[u] >> vshift) & vmask);
        if (pflag && pflag[u]) poffs[ppos[u]] = p;  // first child of the parent entry
    }
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

// --- annotations -----------------------------------------------------------

__device__ __forceinline__ double anno_load(const void *col, uint32_t type, uint32_t row) {
    switch (type) {
        case LH_T_F32: return (double)((const float *)col)[row];
        case LH_T_F64: return ((const double *)col)[row];
        case LH_T_I8: return (double)((const int8_t *)col)[row];
        case LH_T_I32: return (double)((const int32_t *)col)[row];
        default: return (double)((const uint32_t *)col)[row];
    }
}

struct AnnoArgs {
    const void *in[LH_MAX_ANNOS];
    uint32_t in_type[LH_MAX_ANNOS];
    void *out[LH_MAX_ANNOS];
    uint32_t nin;
    uint32_t merge;
};

// One thread per distinct tuple merges the rows of its run (sorted row ids
// rid[runstart[u] .. runstart[u+1])) in sorted order.
__global__ void k_annos(AnnoArgs a, const uint32_t *rid, const uint64_t *runstart, uint64_t nu,
                        uint64_t n) {
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu;
         u += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t r0 = runstart[u], r1 = (u + 1 < nu) ? runstart[u + 1] : n;
        if (a.merge == LH_MERGE_PRICE_DISCOUNT) {
            // expression annotation price * (1 - d/100) as a compensated pair
            float sh = 0.f, sl = 0.f;
            for (uint64_t r = r0; r < r1; ++r) {
                uint32_t row = rid[r];
                float p = (float)anno_load(a.in[0], a.in_type[0], row);
                float d = (float)anno_load(a.in[1], a.in_type[1], row);
                float f = (100.f - d) / 100.f;
                float ph, pl;
                lh_two_prod(p, f, ph, pl);
                lh_pair_add(sh, sl, ph, pl);
            }
            float h = sh + sl;
            ((float *)a.out[0])[u] = h;
            ((float *)a.out[1])[u] = sl - (h - sh);
        } else {
            for (uint32_t c = 0; c < a.nin; ++c) {
                uint32_t t = a.in_type[c];
                if (a.merge == LH_MERGE_FIRST) {
                    uint32_t row = rid[r0];
                    switch (t) {
                        case LH_T_F32: ((float *)a.out[c])[u] = ((const float *)a.in[c])[row]; break;
                        case LH_T_F64: ((double *)a.out[c])[u] = ((const double *)a.in[c])[row]; break;
                        case LH_T_I8: ((int8_t *)a.out[c])[u] = ((const int8_t *)a.in[c])[row]; break;
                        default: ((uint32_t *)a.out[c])[u] = ((const uint32_t *)a.in[c])[row]; break;
                    }
                } else if (t == LH_T_F32) {
                    float s = 0.f;
                    for (uint64_t r = r0; r < r1; ++r) s += ((const float *)a.in[c])[rid[r]];
                    ((float *)a.out[c])[u] = s;
                } else {  // f64
                    double s = 0.0;
                    for (uint64_t r = r0; r < r1; ++r) s += ((const double *)a.in[c])[rid[r]];
                    ((double *)a.out[c])[u] = s;
                }
            }
        }
    }
}

size_t dtype_size(uint32_t t) {
    switch (t) {
        case LH_T_F64: return 8;
        case LH_T_I8: return 1;
        default: return 4;
    }
}

// --- layout ---------------------------------------------------------------

// Per set: decide bitset and its word count (0 = uint layout).
__global__ void k_layout_decide(const uint32_t *vals, const uint32_t *poffs, uint64_t nsets,
                                uint32_t n0, uint32_t ratio, uint32_t min_card, uint32_t *is_bs,
                                uint64_t *nwords) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsets;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = poffs ? poffs[s] : 0, hi = poffs ? poffs[s + 1] : n0;
        uint32_t card = hi - lo;
        uint32_t bs = 0;
        uint64_t w = 0;
        if (ratio > 0 && card >= min_card && card > 0) {
            uint32_t mn = vals[lo], mx = vals[hi - 1];
            uint64_t span = (uint64_t)mx - mn + 1;
            if ((uint64_t)card * ratio >= span) {
                uint32_t base = mn & ~127u;
                w = (((uint64_t)mx - base) >> 5) + 1;
                w = (w + 3) & ~3ull;
                bs = 1;
            }
        }
        is_bs[s] = bs;
        nwords[s] = w;
    }
}

__global__ void k_layout_fill(const uint32_t *vals, const uint32_t *poffs, uint64_t nsets,
                              uint32_t n0, const uint32_t *is_bs, const uint32_t *slot_of,
                              const uint64_t *word_off, uint64_t word_base, uint32_t *bs_slot,
                              uint32_t *bs_meta, uint32_t *slot_set) {
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsets;
         s += (uint64_t)gridDim.x * blockDim.x) {
        if (!is_bs[s]) {
            bs_slot[s] = LH_NOSLOT;
            continue;
        }
        uint32_t lo = poffs ? poffs[s] : 0, hi = poffs ? poffs[s + 1] : n0;
        uint32_t slot = slot_of[s];
        uint64_t w0 = word_base + word_off[s];
        uint64_t nw = word_off[s + 1] - word_off[s];
        bs_slot[s] = slot;
        bs_meta[4 * (uint64_t)slot + 0] = (uint32_t)w0;
        bs_meta[4 * (uint64_t)slot + 1] = vals[lo] & ~127u;
        bs_meta[4 * (uint64_t)slot + 2] = (uint32_t)nw;
        bs_meta[4 * (uint64_t)slot + 3] = hi - lo;
        slot_set[slot] = (uint32_t)s;
    }
}

// Bits of the bitset sets, element-parallel: every bitset set is cut into
// chunks of kBitsChunk elements, one block per chunk, 8 consecutive elements
// per thread; a thread ORs the bits that fall in one word and issues one
// atomicOr per word it touches.
constexpr uint32_t kBitsChunk = 2048;

__global__ void k_layout_chunks(const uint32_t *bs_meta, uint64_t n_bs, uint32_t *chunks) {
    for (uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < n_bs;
         slot += (uint64_t)gridDim.x * blockDim.x)
        chunks[slot] = (bs_meta[4 * slot + 3] + kBitsChunk - 1) / kBitsChunk;  // field 3 = card here
}

__global__ void __launch_bounds__(256) k_layout_bits(const uint32_t *vals, const uint32_t *poffs, uint32_t n0,
                                                     const uint32_t *bs_meta, const uint32_t *slot_set,
                                                     const uint32_t *chunk_off, uint32_t n_bs,
                                                     uint32_t *words) {
    const uint32_t total = chunk_off[n_bs];
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        uint32_t lo_s = 0, hi_s = n_bs;  // chunk_off[lo_s] <= c < chunk_off[hi_s]
        while (hi_s - lo_s > 1) {
            uint32_t mid = (lo_s + hi_s) >> 1;
            if (chunk_off[mid] <= c) lo_s = mid;
            else hi_s = mid;
        }
        const uint32_t slot = lo_s;
        const uint32_t s = slot_set[slot];
        const uint32_t lo = poffs ? poffs[s] : 0, hi = poffs ? poffs[s + 1] : n0;
        const uint32_t w0 = bs_meta[4 * slot + 0], base = bs_meta[4 * slot + 1];
        const uint32_t q0 = lo + (c - chunk_off[slot]) * kBitsChunk + threadIdx.x * 8;
        const uint32_t q1 = min(q0 + 8, hi);
        uint32_t cur = 0xFFFFFFFFu, mask = 0;
        for (uint32_t q = q0; q < q1; ++q) {
            const uint32_t d = vals[q] - base;
            const uint32_t w = d >> 5;
            if (w != cur) {
                if (mask) atomicOr(&words[w0 + cur], mask);
                cur = w;
                mask = 0;
            }
            mask |= 1u << (d & 31u);
        }
        if (mask) atomicOr(&words[w0 + cur], mask);
    }
}

__global__ void k_popc_words(const uint32_t *words, uint64_t n, uint32_t *pc) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        pc[i] = __popc(words[i]);
}

// bs_meta field 3 <- rank of the set's first word (rank is arena-wide)
__global__ void k_rank_base(uint32_t *bs_meta, uint64_t n_bs, const uint32_t *rank) {
    for (uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < n_bs;
         slot += (uint64_t)gridDim.x * blockDim.x)
        bs_meta[4 * slot + 3] = rank[bs_meta[4 * slot + 0]];
}

}  // namespace

// ------------------------------------------------------------------- helpers

void lh_trie_release(lh_ctx *ctx, lh_trie *t) {
    if (!t) return;
    for (void *p : t->allocs) lh_free(ctx, p);
    t->allocs.clear();
}

template <class T>
static lh_status trie_alloc(lh_ctx *ctx, lh_trie *t, T **p, size_t count) {
    LH_TRY(lh_alloc(ctx, p, count));
    t->allocs.push_back((void *)*p);
    t->bytes += (count ? count : 1) * sizeof(T);
    return LH_OK;
}

DTrie lh_trie_dview(const lh_trie *t) {
    DTrie d;
    memset(&d, 0, sizeof(d));
    d.nlevels = t->nlevels;
    for (uint32_t l = 0; l < t->nlevels; ++l) {
        d.lv[l].vals = t->lv[l].vals;
        d.lv[l].offs = t->lv[l].offs;
        d.lv[l].bs_slot = t->lv[l].bs_slot;
        d.lv[l].bs_meta = (const uint4 *)t->lv[l].bs_meta;
        d.lv[l].n = (uint32_t)t->lv[l].n;
    }
    d.words = t->words;
    d.rank = t->rank;
    return d;
}

lh_status lh_trie_layout(lh_ctx *ctx, lh_trie *t) {
    const unsigned T = 256;
    uint64_t total_words = 0;
    uint64_t level_word_base[LH_MAX_LEVELS] = {0};
    std::vector<uint32_t *> tmp_isbs(t->nlevels, nullptr), tmp_slot(t->nlevels, nullptr);
    std::vector<uint64_t *> tmp_words(t->nlevels, nullptr), tmp_woff(t->nlevels, nullptr);
    std::vector<uint32_t *> slot_set(t->nlevels, nullptr);
    lh_status s = LH_OK;
    auto cleanup = [&]() {
        for (uint32_t l = 0; l < t->nlevels; ++l) {
            lh_free(ctx, tmp_isbs[l]);
            lh_free(ctx, tmp_slot[l]);
            lh_free(ctx, tmp_words[l]);
            lh_free(ctx, tmp_woff[l]);
            lh_free(ctx, slot_set[l]);
        }
    };
    for (uint32_t l = 0; l < t->nlevels && s == LH_OK; ++l) {
        TrieLevel &L = t->lv[l];
        L.nsets = (l == 0) ? 1 : t->lv[l - 1].n;
        L.n_bs = 0;
        if (t->bs_ratio == 0 || L.n == 0) continue;
        const uint32_t *poffs = (l == 0) ? nullptr : t->lv[l - 1].offs;
        uint32_t n0 = (uint32_t)L.n;
        if ((s = lh_alloc(ctx, &tmp_isbs[l], L.nsets)) != LH_OK) break;
        if ((s = lh_alloc(ctx, &tmp_slot[l], L.nsets + 1)) != LH_OK) break;
        if ((s = lh_alloc(ctx, &tmp_words[l], L.nsets)) != LH_OK) break;
        if ((s = lh_alloc(ctx, &tmp_woff[l], L.nsets + 1)) != LH_OK) break;
        LH_TRACED(ctx, "k_layout_decide", k_layout_decide<<<lh_blocks(L.nsets, T, 1 << 16), T, 0, ctx->stream>>>(
            L.vals, poffs, L.nsets, n0, t->bs_ratio, t->bs_min_card, tmp_isbs[l], tmp_words[l]));
        if ((s = lh_scan_u32_to_u32(ctx, tmp_isbs[l], tmp_slot[l], L.nsets)) != LH_OK) break;
        if ((s = lh_scan_u64_to_u64(ctx, tmp_words[l], tmp_woff[l], L.nsets)) != LH_OK) break;
        uint32_t nbs = 0;
        uint64_t nw = 0;
        if ((s = lh_readback(ctx, tmp_slot[l] + L.nsets, sizeof(uint32_t), &nbs)) != LH_OK) break;
        if ((s = lh_readback(ctx, tmp_woff[l] + L.nsets, sizeof(uint64_t), &nw)) != LH_OK) break;
        L.n_bs = nbs;
        level_word_base[l] = total_words;
        total_words += nw;
    }
    // ranks are 32-bit: the arena's bit count must stay below 2^32
    if (s == LH_OK && total_words >= (1ull << 27))
        s = lh_fail(ctx, LH_EOVERFLOW, "bitset arena exceeds 2^27 words");
    if (s == LH_OK && total_words > 0) {
        t->nwords = total_words;
        s = trie_alloc(ctx, t, &t->words, total_words);
        if (s == LH_OK) s = trie_alloc(ctx, t, &t->rank, total_words);
        if (s == LH_OK) {
            cudaError_t e = cudaMemsetAsync(t->words, 0, total_words * 4, ctx->stream);
            if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "memset: %s", cudaGetErrorString(e));
        }
    }
    for (uint32_t l = 0; l < t->nlevels && s == LH_OK; ++l) {
        TrieLevel &L = t->lv[l];
        if (L.n_bs == 0) continue;
        const uint32_t *poffs = (l == 0) ? nullptr : t->lv[l - 1].offs;
        uint32_t n0 = (uint32_t)L.n;
        if ((s = trie_alloc(ctx, t, &L.bs_slot, L.nsets)) != LH_OK) break;
        if ((s = trie_alloc(ctx, t, &L.bs_meta, 4 * L.n_bs)) != LH_OK) break;
        if ((s = lh_alloc(ctx, &slot_set[l], L.n_bs)) != LH_OK) break;
        LH_TRACED(ctx, "k_layout_fill", k_layout_fill<<<lh_blocks(L.nsets, T, 1 << 16), T, 0, ctx->stream>>>(
            L.vals, poffs, L.nsets, n0, tmp_isbs[l], tmp_slot[l], tmp_woff[l], level_word_base[l],
            L.bs_slot, L.bs_meta, slot_set[l]));
        uint32_t *chunks = nullptr, *coff = nullptr;
        if ((s = lh_alloc(ctx, &chunks, L.n_bs)) != LH_OK) break;
        if ((s = lh_alloc(ctx, &coff, L.n_bs + 1)) != LH_OK) { lh_free(ctx, chunks); break; }
        LH_TRACED(ctx, "k_layout_chunks", k_layout_chunks<<<lh_blocks(L.n_bs, T, 1 << 16), T, 0, ctx->stream>>>(
            L.bs_meta, L.n_bs, chunks));
        s = lh_scan_u32_to_u32(ctx, chunks, coff, L.n_bs);
        uint32_t nch = 0;
        if (s == LH_OK) s = lh_readback(ctx, coff + L.n_bs, sizeof(uint32_t), &nch);
        if (s == LH_OK && nch)
            LH_TRACED(ctx, "k_layout_bits", k_layout_bits<<<std::min<uint32_t>(nch, (uint32_t)ctx->num_sms * 16), 256, 0, ctx->stream>>>(
                L.vals, poffs, n0, L.bs_meta, slot_set[l], coff, (uint32_t)L.n_bs, t->words));
        lh_free(ctx, chunks);
        lh_free(ctx, coff);
        cudaError_t e = cudaGetLastError();
        if (s == LH_OK && e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "layout: %s", cudaGetErrorString(e));
    }
    // arena-wide exclusive rank of every word, then each set's rank base
    if (s == LH_OK && total_words > 0) {
        uint32_t *pc = nullptr;
        s = lh_alloc(ctx, &pc, total_words);
        if (s == LH_OK) {
            LH_TRACED(ctx, "k_popc_words", k_popc_words<<<lh_blocks(total_words, T, (uint32_t)ctx->num_sms * 16), T, 0, ctx->stream>>>(
                t->words, total_words, pc));
            s = lh_scan_u32_to_u32(ctx, pc, t->rank, total_words - 1);
        }
        lh_free(ctx, pc);
        for (uint32_t l = 0; l < t->nlevels && s == LH_OK; ++l)
            if (t->lv[l].n_bs)
                LH_TRACED(ctx, "k_rank_base", k_rank_base<<<lh_blocks(t->lv[l].n_bs, T, 1 << 16), T, 0, ctx->stream>>>(
                    t->lv[l].bs_meta, t->lv[l].n_bs, t->rank));
    }
    cleanup();
    return s;
}

// -------------------------------------------------------------- C ABI entry

extern "C" lh_status lh_build_trie(lh_ctx *ctx, const lh_relation_desc *rel,
                                   const uint32_t *key_order, const lh_layout_policy *layout,
                                   lh_merge merge, lh_trie **out) {
    if (!ctx || !rel || !out || !key_order) return lh_fail(ctx, LH_EINVAL, "null argument");
    *out = nullptr;
    const uint32_t L = rel->nkeys;
    if (L == 0 || L > LH_MAX_LEVELS) return lh_fail(ctx, LH_EINVAL, "nkeys must be 1..%d", LH_MAX_LEVELS);
    if (rel->nrows >= (1ull << 32)) return lh_fail(ctx, LH_EOVERFLOW, "more than 2^32-1 rows");
    bool seen[LH_MAX_LEVELS] = {false};
    for (uint32_t l = 0; l < L; ++l) {
        if (key_order[l] >= L || seen[key_order[l]])
            return lh_fail(ctx, LH_EINVAL, "key_order is not a permutation");
        seen[key_order[l]] = true;
        if (!rel->keys[key_order[l]] && rel->nrows) return lh_fail(ctx, LH_EINVAL, "null key column");
    }
    if (rel->nannos > LH_MAX_ANNOS) return lh_fail(ctx, LH_EINVAL, "too many annotation columns");
    if (merge == LH_MERGE_PRICE_DISCOUNT) {
        if (rel->nannos != 2 || rel->anno_types[1] != LH_T_I8 ||
            (rel->anno_types[0] != LH_T_F64 && rel->anno_types[0] != LH_T_F32))
            return lh_fail(ctx, LH_EINVAL, "price/discount merge needs (f32|f64 price, i8 discount)");
    } else if (merge == LH_MERGE_SUM) {
        for (uint32_t c = 0; c < rel->nannos; ++c)
            if (rel->anno_types[c] != LH_T_F32 && rel->anno_types[c] != LH_T_F64)
                return lh_fail(ctx, LH_EINVAL, "sum merge needs float annotation columns");
    } else if (merge != LH_MERGE_FIRST) {
        return lh_fail(ctx, LH_EINVAL, "unknown merge");
    }
    lh_layout_policy pol = layout ? *layout : lh_layout_policy{32, 32};

    lh_trie *t = new lh_trie();
    t->nlevels = L;
    t->nrows_in = rel->nrows;
    t->bs_ratio = pol.bs_ratio;
    t->bs_min_card = pol.bs_min_card;
    for (uint32_t l = 0; l < L; ++l) t->key_order[l] = key_order[l];
    const uint64_t n = rel->nrows;
    const unsigned T = 256;
    const unsigned G = (unsigned)std::min<uint64_t>(lh_blocks(n, T), (uint64_t)ctx->num_sms * 16);

    uint32_t *d_max = nullptr;
    uint64_t *key = nullptr, *tkey = nullptr, *ukey = nullptr, *runstart = nullptr, *upos = nullptr;
    uint32_t *rid = nullptr, *trid = nullptr, *flag = nullptr;
    std::vector<uint32_t *> lflag(L, nullptr), lpos(L, nullptr);
    uint64_t nu = 0;
    lh_status s = LH_OK;
    auto cleanup_tmp = [&]() {
        lh_free(ctx, d_max); lh_free(ctx, key); lh_free(ctx, tkey); lh_free(ctx, ukey);
        lh_free(ctx, runstart); lh_free(ctx, upos); lh_free(ctx, rid); lh_free(ctx, trid);
        lh_free(ctx, flag);
        for (uint32_t l = 0; l < L; ++l) { lh_free(ctx, lflag[l]); lh_free(ctx, lpos[l]); }
    };
#define STEP(x) if (s == LH_OK) s = (x)
    // 1. key widths
    uint32_t bits[LH_MAX_LEVELS] = {0};
    uint32_t total_bits = 0;
    STEP(lh_alloc(ctx, &d_max, L));
    if (s == LH_OK) {
        cudaMemsetAsync(d_max, 0, L * sizeof(uint32_t), ctx->stream);
        for (uint32_t l = 0; l < L && n; ++l)
            LH_TRACED(ctx, "k_col_max", k_col_max<<<G, T, 0, ctx->stream>>>(rel->keys[key_order[l]], n, d_max + l));
        uint32_t hmax[LH_MAX_LEVELS] = {0};
        STEP(lh_readback(ctx, d_max, L * sizeof(uint32_t), hmax));
        for (uint32_t l = 0; l < L; ++l) {
            bits[l] = hmax[l] ? 32 - __builtin_clz(hmax[l]) : 1;
            t->key_bits[l] = bits[l];
            total_bits += bits[l];
        }
        if (s == LH_OK && total_bits > 64)
            s = lh_fail(ctx, LH_EUNSUPPORTED, "packed key needs %u > 64 bits", total_bits);
    }
    // 2. pack + sort
    PackArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.nlev = L;
    uint32_t shift[LH_MAX_LEVELS];
    {
        uint32_t acc = 0;
        for (int l = (int)L - 1; l >= 0; --l) {  // level 0 most significant
            shift[l] = acc;
            acc += bits[l];
        }
        for (uint32_t l = 0; l < L; ++l) {
            pa.col[l] = rel->keys[key_order[l]];
            pa.shift[l] = shift[l];
        }
    }
    STEP(lh_alloc(ctx, &key, n));
    STEP(lh_alloc(ctx, &tkey, n));
    STEP(lh_alloc(ctx, &rid, n));
    STEP(lh_alloc(ctx, &trid, n));
    STEP(lh_alloc(ctx, &flag, n));
    STEP(lh_alloc(ctx, &upos, n + 1));
    if (s == LH_OK && n) {
        LH_TRACED(ctx, "k_pack", k_pack<<<G, T, 0, ctx->stream>>>(pa, n, key, rid));
        STEP(lh_radix_sort_u64(ctx, key, rid, tkey, trid, n, (int)total_bits));
        if (s == LH_OK) LH_TRACED(ctx, "k_heads", k_heads<<<G, T, 0, ctx->stream>>>(key, n, flag));
        STEP(lh_scan_u32_to_u64(ctx, flag, upos, n));
        STEP(lh_readback(ctx, upos + n, sizeof(uint64_t), &nu));
    }
    STEP(lh_alloc(ctx, &ukey, nu));
    STEP(lh_alloc(ctx, &runstart, nu));
    if (s == LH_OK && n) LH_TRACED(ctx, "k_compact_unique", k_compact_unique<<<G, T, 0, ctx->stream>>>(key, flag, upos, n, ukey, runstart));
    // 3. levels
    for (uint32_t l = 0; l < L && s == LH_OK; ++l) {
        STEP(lh_alloc(ctx, &lflag[l], nu));
        STEP(lh_alloc(ctx, &lpos[l], nu + 1));
        if (s != LH_OK) break;
        if (nu) LH_TRACED(ctx, "k_level_flags", k_level_flags<<<G, T, 0, ctx->stream>>>(ukey, nu, shift[l], lflag[l]));
        STEP(lh_scan_u32_to_u32(ctx, lflag[l], lpos[l], nu));
        uint32_t nl = 0;
        STEP(lh_readback(ctx, lpos[l] + nu, sizeof(uint32_t), &nl));
        t->lv[l].n = nu ? nl : 0;
    }
    for (uint32_t l = 0; l < L && s == LH_OK; ++l) {
        TrieLevel &lv = t->lv[l];
        STEP(trie_alloc(ctx, t, &lv.vals, lv.n));
        if (l + 1 < L) STEP(trie_alloc(ctx, t, &lv.offs, lv.n + 1));
    }
    for (uint32_t l = 0; l < L && s == LH_OK; ++l) {
        uint64_t vmask = (bits[l] >= 64) ? ~0ull : ((1ull << bits[l]) - 1);
        if (nu)
            LH_TRACED(ctx, "k_level_emit", k_level_emit<<<G, T, 0, ctx->stream>>>(
                ukey, nu, lflag[l], lpos[l], shift[l], vmask, t->lv[l].vals,
                l ? lflag[l - 1] : nullptr, l ? lpos[l - 1] : nullptr, l ? t->lv[l - 1].offs : nullptr));
        if (l + 1 < L) LH_TRACED(ctx, "k_set_u32", k_set_u32<<<1, 1, 0, ctx->stream>>>(t->lv[l].offs + t->lv[l].n, (uint32_t)t->lv[l + 1].n));
    }
    // 4. annotations in leaf order
    if (s == LH_OK && rel->nannos) {
        AnnoArgs aa;
        memset(&aa, 0, sizeof(aa));
        aa.merge = merge;
        aa.nin = rel->nannos;
        for (uint32_t c = 0; c < rel->nannos; ++c) {
            aa.in[c] = rel->annos[c];
            aa.in_type[c] = rel->anno_types[c];
        }
        if (merge == LH_MERGE_PRICE_DISCOUNT) {
            t->nannos = 2;
            for (int c = 0; c < 2 && s == LH_OK; ++c) {
                float *p = nullptr;
                STEP(trie_alloc(ctx, t, &p, nu));
                t->anno[c] = p;
                t->anno_type[c] = LH_T_F32;
                aa.out[c] = p;
            }
        } else {
            t->nannos = rel->nannos;
            for (uint32_t c = 0; c < rel->nannos && s == LH_OK; ++c) {
                uint8_t *p = nullptr;
                STEP(trie_alloc(ctx, t, &p, nu * dtype_size(rel->anno_types[c])));
                t->anno[c] = p;
                t->anno_type[c] = rel->anno_types[c];
                aa.out[c] = p;
            }
        }
        if (s == LH_OK && nu) LH_TRACED(ctx, "k_annos", k_annos<<<G, T, 0, ctx->stream>>>(aa, rid, runstart, nu, n));
    }
    if (s == LH_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "build_trie: %s", cudaGetErrorString(e));
    }
    cleanup_tmp();
    STEP(lh_trie_layout(ctx, t));
#undef STEP
    if (s != LH_OK) {
        lh_trie_release(ctx, t);
        delete t;
        return s;
    }
    *out = t;
    return LH_OK;
}

namespace {
__global__ void k_filter_flags(const int32_t *col, uint64_t n, int32_t lo, int32_t hi, uint32_t *flag) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        int32_t v = col[i];
        flag[i] = (v >= lo && v <= hi) ? 1u : 0u;
    }
}
__global__ void k_filter_emit(const uint32_t *flag, const uint32_t *pos, uint64_t n, uint32_t *vals) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (flag[i]) vals[pos[i]] = (uint32_t)i;
}
}  // namespace

extern "C" lh_status lh_filter_trie(lh_ctx *ctx, const int32_t *col, uint64_t n, int32_t lo, int32_t hi,
                                    const lh_layout_policy *layout, lh_trie **out) {
    if (!ctx || !out || (!col && n)) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (n >= (1ull << 32)) return lh_fail(ctx, LH_EOVERFLOW, "more than 2^32-1 keys");
    *out = nullptr;
    lh_layout_policy pol = layout ? *layout : lh_layout_policy{32, 32};
    lh_trie *t = new lh_trie();
    t->nlevels = 1;
    t->nrows_in = n;
    t->key_bits[0] = n > 1 ? 64 - __builtin_clzll(n - 1) : 1;
    t->bs_ratio = pol.bs_ratio;
    t->bs_min_card = pol.bs_min_card;
    const unsigned T = 256;
    const unsigned G = (unsigned)std::min<uint64_t>(lh_blocks(n, T), (uint64_t)ctx->num_sms * 16);
    uint32_t *flag = nullptr, *pos = nullptr;
    lh_status s = lh_alloc(ctx, &flag, n);
    if (s == LH_OK) s = lh_alloc(ctx, &pos, n + 1);
    if (s == LH_OK && n) LH_TRACED(ctx, "k_filter_flags", k_filter_flags<<<G, T, 0, ctx->stream>>>(col, n, lo, hi, flag));
    if (s == LH_OK) s = lh_scan_u32_to_u32(ctx, flag, pos, n);
    uint32_t cnt = 0;
    if (s == LH_OK) s = lh_readback(ctx, pos + n, sizeof(uint32_t), &cnt);
    t->lv[0].n = cnt;
    if (s == LH_OK) s = trie_alloc(ctx, t, &t->lv[0].vals, cnt);
    if (s == LH_OK && n) LH_TRACED(ctx, "k_filter_emit", k_filter_emit<<<G, T, 0, ctx->stream>>>(flag, pos, n, t->lv[0].vals));
    lh_free(ctx, flag);
    lh_free(ctx, pos);
    if (s == LH_OK) s = lh_trie_layout(ctx, t);
    if (s != LH_OK) {
        lh_trie_release(ctx, t);
        delete t;
        return s;
    }
    *out = t;
    return LH_OK;
}

extern "C" lh_status lh_trie_free(lh_ctx *ctx, lh_trie *t) {
    if (!ctx || !t) return LH_EINVAL;
    lh_trie_release(ctx, t);
    delete t;
    return LH_OK;
}

extern "C" lh_status lh_trie_stats_get(lh_ctx *ctx, const lh_trie *t, lh_trie_stats *o) {
    if (!ctx || !t || !o) return lh_fail(ctx, LH_EINVAL, "null argument");
    memset(o, 0, sizeof(*o));
    o->nlevels = t->nlevels;
    o->nrows_in = t->nrows_in;
    for (uint32_t l = 0; l < t->nlevels; ++l) {
        o->key_order[l] = t->key_order[l];
        o->level_n[l] = t->lv[l].n;
        o->level_sets[l] = (l == 0) ? 1 : t->lv[l - 1].n;
        o->level_bs_sets[l] = t->lv[l].n_bs;
    }
    o->bitset_words = t->nwords;
    o->device_bytes = t->bytes;
    return LH_OK;
}

extern "C" lh_status lh_trie_level(lh_ctx *ctx, const lh_trie *t, uint32_t level, lh_level_view *o) {
    if (!ctx || !t || !o) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (level >= t->nlevels) return lh_fail(ctx, LH_EINVAL, "level out of range");
    const TrieLevel &L = t->lv[level];
    o->n = L.n;
    o->nsets = (level == 0) ? 1 : t->lv[level - 1].n;
    o->vals = L.vals;
    o->child_offs = L.offs;
    o->bs_slot = L.bs_slot;
    o->n_bs = L.n_bs;
    o->bs_meta = L.bs_meta;
    o->words = t->words;
    o->rank = t->rank;
    return LH_OK;
}

extern "C" lh_status lh_trie_anno(lh_ctx *ctx, const lh_trie *t, uint32_t col, const void **ptr,
                                  uint32_t *dtype) {
    if (!ctx || !t || !ptr || !dtype) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (col >= t->nannos) return lh_fail(ctx, LH_EINVAL, "annotation column out of range");
    *ptr = t->anno[col];
    *dtype = t->anno_type[col];
    return LH_OK;
}
