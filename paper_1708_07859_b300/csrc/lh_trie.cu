// Trie construction (Section 2.2): key tuples packed in attribute order,
// radix-sorted, deduplicated with annotation merge, emitted as CSR levels;
// each set then gets the uint or bitset layout; annotations are gathered into
// leaf order (Section 3.1: each annotation in its own buffer).  Also the
// filter relation of a pushed-down selection (Section 3.2).
#include "lh_internal.cuh"

namespace {

struct PackArgs {
    const uint32_t *col[LH_MAX_LEVELS];
    uint32_t shift[LH_MAX_LEVELS];
    uint32_t bound[LH_MAX_LEVELS];  // declared domain sizes checked while packing, 0 = none
    uint32_t nlev;
    const uint32_t *payload;  // 4-byte annotation carried through the sort, or null: row ids
    uint32_t *status;         // LH_EINVAL when a value breaks its bound
    unsigned long long *hist; // digit counts of every sort pass (pass p at hist[256 p]), zeroed
    int passes;
};

// Largest value of every key column, one launch: each thread takes four
// rows per grid stride, all loads issued before the maxima.
__global__ void k_col_max(PackArgs a, uint64_t n, uint32_t *out) {
    uint32_t m[LH_MAX_LEVELS] = {0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
#pragma unroll
        for (int l = 0; l < LH_MAX_LEVELS; ++l) {
            if (l >= (int)a.nlev) break;
            uint32_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = i + u * stride < n ? a.col[l][i + u * stride] : 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) m[l] = max(m[l], v[u]);
        }
    }
#pragma unroll
    for (int l = 0; l < LH_MAX_LEVELS; ++l) {
        if (l >= (int)a.nlev) break;
        uint32_t x = m[l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(LH_FULL, x, o));
        if ((threadIdx.x & 31) == 0) atomicMax(out + l, x);
    }
}

// Packed key (level 0 in the high bits) and sort payload of every row; four
// rows per thread and grid stride, loaded before they are stored.
__global__ void k_pack(PackArgs a, uint64_t n, uint64_t *key, uint32_t *rid) {
    // the radix sort's digit counts of every pass, counted while the keys are
    // in registers (per-block shared histograms, folded into a.hist at the end)
    __shared__ uint32_t h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
        uint64_t k[4] = {0, 0, 0, 0};
        uint32_t r[4];
        bool bad = false;
#pragma unroll
        for (int l = 0; l < LH_MAX_LEVELS; ++l) {
            if (l >= (int)a.nlev) break;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + u * stride < n) {
                    const uint32_t v = a.col[l][i + u * stride];
                    bad |= a.bound[l] != 0 && v >= a.bound[l];
                    k[u] |= (uint64_t)v << a.shift[l];
                }
        }
        if (bad) lh_set_status(a.status, LH_EINVAL);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            r[u] = i + u * stride < n ? (a.payload ? a.payload[i + u * stride] : (uint32_t)(i + u * stride)) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i + u * stride < n) {
                key[i + u * stride] = k[u];
                rid[i + u * stride] = r[u];
                for (int p = 0; p < a.passes; ++p) atomicAdd(&h[p][(k[u] >> (8 * p)) & 255u], 1u);
            }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(a.hist + i, (unsigned long long)c);
    }
}

// ---- CSR levels from the sorted packed keys, in one pass ------------------
// Level l's prefix of key k is k >> shift[l] (levels 0..l); a sorted row i
// opens a level-l entry when that prefix differs from row i-1's.  A tile of
// 4096 rows (2048 beyond three levels) is staged in shared memory; thread t
// takes rows j * 256 + t, so the entries a warp opens for one j land at
// consecutive indices (ballot + popc) and its stores coalesce.  Warp l scans the tile's per-(j, warp)
// counts of level l, finds the tile's offset in level l by decoupled
// look-back over tile tickets, and then every opened entry writes its value,
// its first child's index in the level below and (leaf level) the first
// sorted row of its distinct key.  Tiles are ticketed in order, so every
// tile a tile waits on is already running and publishes its count without
// waiting.
constexpr int kLvThreads = 256;
constexpr int kLvWarps = kLvThreads / 32;
// rows per thread: 16 (4096-row tiles) for up to three levels, 8 beyond,
// where the per-level ballot words would spill
__host__ __device__ constexpr int lv_items(int nl) { return nl <= 3 ? 16 : 8; }
__host__ __device__ constexpr uint64_t lv_tile(int nl) { return (uint64_t)kLvThreads * lv_items(nl); }
constexpr unsigned long long kLvAgg = 1ull << 62, kLvInc = 1ull << 63, kLvVal = (1ull << 62) - 1;
constexpr uint32_t kLvSpins = 1u << 20;

struct LevelArgs {
    uint32_t nlev;
    uint32_t shift[LH_MAX_LEVELS];
    uint32_t vmask[LH_MAX_LEVELS];
    uint32_t *vals[LH_MAX_LEVELS];  // capacity n each
    uint32_t *offs[LH_MAX_LEVELS];  // levels 0..nlev-2, capacity n + 1 each
    uint32_t *runstart;             // capacity n
    unsigned long long *state;      // [tiles][nlev], zeroed
    uint32_t *ticket;               // zeroed
    uint64_t *count;                // [nlev]: entries per level
    uint32_t *status;
};

__device__ __forceinline__ void lv_store(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long lv_load(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <int NL>
__global__ void __launch_bounds__(kLvThreads) k_levels(const uint64_t *key, uint64_t n, LevelArgs a) {
    constexpr int kLvItems = lv_items(NL);
    constexpr uint64_t kLvTile = lv_tile(NL);
    constexpr int kPer = kLvItems * kLvWarps / 32;  // (j, warp) counts per lane in the scan
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_ok;
    __shared__ uint64_t s_k[kLvTile];
    __shared__ uint32_t s_base[NL][kLvItems * kLvWarps];  // per (j, warp) counts, then exclusive bases
    __shared__ uint64_t s_agg[NL];
    __shared__ uint64_t s_off[NL];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    if (t == 0) {
        s_tile = atomicAdd(a.ticket, 1u);
        s_ok = 1;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t tb = (uint64_t)tile * kLvTile;
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) {
        const uint32_t r = j * kLvThreads + t;
        s_k[r] = tb + r < n ? key[tb + r] : 0;
    }
    const uint64_t before_tile = (tb > 0 && tb <= n) ? key[tb - 1] : 0;
    __syncthreads();
    // bal[l][j] bit lane: row j * 256 + 32 * warp + lane opens a level-l entry
    uint32_t bal[NL][kLvItems];
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) {
        const uint32_t r = j * kLvThreads + t;
        const uint64_t i = tb + r;
        const uint64_t k = s_k[r], pk = r ? s_k[r - 1] : before_tile;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const bool open = i < n && (i == 0 || (k >> a.shift[l]) != (pk >> a.shift[l]));
            bal[l][j] = __ballot_sync(LH_FULL, open);
            if (lane == 0) s_base[l][j * kLvWarps + warp] = __popc(bal[l][j]);
        }
    }
    __syncthreads();
    if (warp < NL) {
        const uint32_t l = warp;
        // exclusive scan of the (j, warp) counts in row order; lane holds kPer
        uint32_t cc[kPer];
        uint32_t mine = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            cc[i] = s_base[l][kPer * lane + i];
            mine += cc[i];
        }
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(LH_FULL, incl, o);
            if (lane >= o) incl += x;
        }
        uint32_t run = incl - mine;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            s_base[l][kPer * lane + i] = run;
            run += cc[i];
        }
        const uint64_t agg = __shfl_sync(LH_FULL, incl, 31);
        // publish the tile's count, then look back for its offset
        if (lane == 0) lv_store(a.state + (uint64_t)tile * NL + l, (tile == 0 ? kLvInc : kLvAgg) | agg);
        uint64_t excl = 0;
        int64_t q = (int64_t)tile - 1;
        uint32_t spins = 0;
        bool ok = true;
        while (q >= 0) {
            const int64_t qi = q - (int64_t)lane;
            const unsigned long long w = qi >= 0 ? lv_load(a.state + (uint64_t)qi * NL + l) : kLvInc;
            const uint32_t inc = __ballot_sync(LH_FULL, (w & kLvInc) != 0);
            const uint32_t ready = __ballot_sync(LH_FULL, (w >> 62) != 0);
            const uint32_t fi = inc ? (uint32_t)__ffs(inc) - 1 : 31u;
            const uint32_t need = fi == 31 ? LH_FULL : ((2u << fi) - 1u);
            if ((ready & need) != need) {
                if (++spins >= kLvSpins) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
                continue;
            }
            uint64_t v = lane <= fi ? (uint64_t)(w & kLvVal) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LH_FULL, v, o);
            excl += v;
            if (inc) break;
            q -= 32;
        }
        if (lane == 0) {
            if (!ok) {
                lh_set_status(a.status, LH_ETIMEOUT);
                s_ok = 0;
            }
            s_off[l] = excl;
            s_agg[l] = agg;
            if (tile > 0) lv_store(a.state + (uint64_t)tile * NL + l, kLvInc | ((excl + agg) & kLvVal));
        }
    }
    __syncthreads();
    if (!s_ok) return;
#pragma unroll
    for (int j = 0; j < kLvItems; ++j) {
        const uint32_t r = j * kLvThreads + t;
        const uint64_t i = tb + r;
        if (i >= n) break;
        const uint64_t k = s_k[r];
        uint64_t pp = 0;  // index of the entry this row opens one level up
        bool popen = false;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const bool open = (bal[l][j] >> lane) & 1u;
            if (open) {
                const uint64_t p = s_off[l] + s_base[l][j * kLvWarps + warp] + __popc(bal[l][j] & lt_mask);
                a.vals[l][p] = (uint32_t)(k >> a.shift[l]) & a.vmask[l];
                if (popen) a.offs[l - 1][pp] = (uint32_t)p;
                if (l + 1 == NL) a.runstart[p] = (uint32_t)i;
                pp = p;
            }
            popen = open;
        }
        if (i + 1 == n) {
            // the last row closes every level: entry counts and the final offsets
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const uint64_t c = s_off[l] + s_agg[l];
                a.count[l] = c;
                if (l > 0) a.offs[l - 1][s_off[l - 1] + s_agg[l - 1]] = (uint32_t)c;
            }
        }
    }
}

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
__global__ void k_annos(AnnoArgs a, const uint32_t *rid, const uint32_t *runstart, uint64_t nu,
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

// Leaf-order annotation when the (single, 4-byte) annotation rode through
// the sort as its payload: run u covers sorted rows runstart[u] ..
// runstart[u+1]; FIRST takes the run's first row (the sort is stable), SUM
// adds the run in row order.
__global__ void k_annos_carried(const uint32_t *payload, const uint32_t *runstart, uint64_t nu, uint64_t n,
                                uint32_t sum_f32, uint32_t *out) {
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu;
         u += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r0 = runstart[u], r1 = (u + 1 < nu) ? runstart[u + 1] : n;
        if (!sum_f32) {
            out[u] = payload[r0];
        } else {
            float s = 0.f;
            for (uint64_t r = r0; r < r1; ++r) s += __uint_as_float(payload[r]);
            out[u] = __float_as_uint(s);
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
// tot[0] += bitset sets of the level, tot[1] += their words
// The level's set count and entry count come from the host (nsets, n0) or,
// when the pointers are given, from the device (the level build's counts).
__global__ void k_layout_decide(const uint32_t *vals, const uint32_t *poffs, uint64_t nsets,
                                uint32_t n0, const uint64_t *d_nsets, const uint64_t *d_n0, uint32_t ratio,
                                uint32_t min_card, uint32_t *is_bs, uint64_t *nwords, unsigned long long *tot) {
    if (d_nsets) nsets = *d_nsets;
    if (d_n0) n0 = (uint32_t)*d_n0;
    unsigned long long my_bs = 0, my_w = 0;
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
        my_bs += bs;
        my_w += w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_bs += __shfl_xor_sync(LH_FULL, my_bs, o);
        my_w += __shfl_xor_sync(LH_FULL, my_w, o);
    }
    if ((threadIdx.x & 31) == 0 && my_bs) {
        atomicAdd(tot, my_bs);
        atomicAdd(tot + 1, my_w);
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

// Layout decisions already taken on the device together with the level
// build (arrays owned by the layout from then on) and their totals.
struct LayoutPre {
    uint32_t *isbs[LH_MAX_LEVELS];
    uint64_t *words[LH_MAX_LEVELS];
    unsigned long long tot[2 * LH_MAX_LEVELS];
};

static lh_status trie_layout(lh_ctx *ctx, lh_trie *t, LayoutPre *pre);

lh_status lh_trie_layout(lh_ctx *ctx, lh_trie *t) { return trie_layout(ctx, t, nullptr); }

static lh_status trie_layout(lh_ctx *ctx, lh_trie *t, LayoutPre *pre) {
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
    // every level decides and counts its bitset sets and words on the device;
    // one readback brings all totals, and only levels with bitset sets go on
    unsigned long long *d_tot = nullptr;
    unsigned long long h_tot[2 * LH_MAX_LEVELS] = {0};
    bool any = false;
    for (uint32_t l = 0; l < t->nlevels; ++l) {
        TrieLevel &L = t->lv[l];
        L.nsets = (l == 0) ? 1 : t->lv[l - 1].n;
        L.n_bs = 0;
        any = any || (t->level_ratio[l] != 0 && L.n != 0);
    }
    if (pre) {
        for (uint32_t l = 0; l < t->nlevels; ++l) {
            tmp_isbs[l] = pre->isbs[l];
            tmp_words[l] = pre->words[l];
            pre->isbs[l] = nullptr;
            pre->words[l] = nullptr;
        }
        memcpy(h_tot, pre->tot, sizeof(h_tot));
        any = false;  // decided and counted already
    }
    if (any) {
        s = lh_alloc(ctx, &d_tot, 2 * LH_MAX_LEVELS);
        if (s == LH_OK) {
            cudaError_t e = cudaMemsetAsync(d_tot, 0, 2 * LH_MAX_LEVELS * sizeof(unsigned long long), ctx->stream);
            if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "layout: %s", cudaGetErrorString(e));
        }
    }
    for (uint32_t l = 0; l < t->nlevels && s == LH_OK && any; ++l) {
        TrieLevel &L = t->lv[l];
        if (t->level_ratio[l] == 0 || L.n == 0) continue;
        const uint32_t *poffs = (l == 0) ? nullptr : t->lv[l - 1].offs;
        if ((s = lh_alloc(ctx, &tmp_isbs[l], L.nsets)) != LH_OK) break;
        if ((s = lh_alloc(ctx, &tmp_words[l], L.nsets)) != LH_OK) break;
        LH_TRACED(ctx, "k_layout_decide", k_layout_decide<<<lh_blocks(L.nsets, T, 1 << 16), T, 0, ctx->stream>>>(
            L.vals, poffs, L.nsets, (uint32_t)L.n, nullptr, nullptr, t->level_ratio[l], t->bs_min_card, tmp_isbs[l],
            tmp_words[l], d_tot + 2 * l));
    }
    if (s == LH_OK && any) s = lh_readback(ctx, d_tot, sizeof(h_tot), h_tot);
    lh_free(ctx, d_tot);
    for (uint32_t l = 0; l < t->nlevels && s == LH_OK; ++l) {
        TrieLevel &L = t->lv[l];
        L.n_bs = h_tot[2 * l];
        level_word_base[l] = total_words;
        total_words += h_tot[2 * l + 1];
        if (L.n_bs == 0) continue;
        // each bitset set's slot and first word: exclusive scans over the sets
        if ((s = lh_alloc(ctx, &tmp_slot[l], L.nsets + 1)) != LH_OK) break;
        if ((s = lh_alloc(ctx, &tmp_woff[l], L.nsets + 1)) != LH_OK) break;
        if ((s = lh_scan_u32_to_u32(ctx, tmp_isbs[l], tmp_slot[l], L.nsets)) != LH_OK) break;
        if ((s = lh_scan_u64_to_u64(ctx, tmp_words[l], tmp_woff[l], L.nsets)) != LH_OK) break;
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
        // the kernel reads its chunk count on the device; the grid only needs
        // a bound (every set has at least one chunk)
        const uint64_t max_chunks = (uint64_t)L.n_bs + (L.n + kBitsChunk - 1) / kBitsChunk;
        if (s == LH_OK)
            LH_TRACED(ctx, "k_layout_bits", k_layout_bits<<<(unsigned)std::min<uint64_t>(max_chunks, (uint64_t)ctx->num_sms * 16), 256, 0, ctx->stream>>>(
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
    bool any_ratio = false;
    for (uint32_t l = 0; l < LH_MAX_LEVELS; ++l) {
        t->level_ratio[l] = pol.per_level ? pol.level_ratio[l] : pol.bs_ratio;
        any_ratio = any_ratio || (l < L && t->level_ratio[l] != 0);
    }
    for (uint32_t l = 0; l < L; ++l) t->key_order[l] = key_order[l];
    const uint64_t n = rel->nrows;
    const unsigned T = 256;
    const unsigned G = (unsigned)std::min<uint64_t>(lh_blocks(n, T), (uint64_t)ctx->num_sms * 16);
    const unsigned G4 = (unsigned)std::min<uint64_t>(lh_blocks((n + 3) / 4, T), (uint64_t)ctx->num_sms * 16);

    LayoutPre pre;
    memset(&pre, 0, sizeof(pre));
    uint32_t *d_max = nullptr, *ticket = nullptr;
    uint64_t *key = nullptr, *tkey = nullptr, *d_count = nullptr;
    unsigned long long *d_hist = nullptr;
    uint32_t *rid = nullptr, *trid = nullptr, *runstart = nullptr;
    unsigned long long *lstate = nullptr;
    std::vector<uint32_t *> tvals(L, nullptr), toffs(L, nullptr);
    uint64_t nu = 0;
    lh_status s = LH_OK;
    auto cleanup_tmp = [&]() {
        lh_free(ctx, d_max); lh_free(ctx, ticket); lh_free(ctx, key); lh_free(ctx, tkey);
        lh_free(ctx, d_count); lh_free(ctx, d_hist); lh_free(ctx, rid); lh_free(ctx, trid); lh_free(ctx, runstart);
        lh_free(ctx, lstate);
        for (uint32_t l = 0; l < L; ++l) { lh_free(ctx, tvals[l]); lh_free(ctx, toffs[l]); }
    };
    auto free_pre = [&]() {
        for (uint32_t l = 0; l < L; ++l) { lh_free(ctx, pre.isbs[l]); lh_free(ctx, pre.words[l]); }
    };
#define STEP(x) if (s == LH_OK) s = (x)
    // 1. key widths
    uint32_t bits[LH_MAX_LEVELS] = {0};
    uint32_t total_bits = 0;
    PackArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.nlev = L;
    for (uint32_t l = 0; l < L; ++l) pa.col[l] = rel->keys[key_order[l]];
    bool bounded = true;
    for (uint32_t l = 0; l < L; ++l) bounded = bounded && rel->key_bound[key_order[l]] != 0;
    if (bounded) {
        // declared domains: widths without reading the columns (k_pack checks them)
        for (uint32_t l = 0; l < L; ++l) {
            const uint32_t b = rel->key_bound[key_order[l]];
            pa.bound[l] = b;
            bits[l] = b > 1 ? 32 - __builtin_clz(b - 1) : 1;
        }
    } else {
        STEP(lh_alloc(ctx, &d_max, L));
        if (s == LH_OK) {
            cudaMemsetAsync(d_max, 0, L * sizeof(uint32_t), ctx->stream);
            if (n) LH_TRACED(ctx, "k_col_max", k_col_max<<<G4, T, 0, ctx->stream>>>(pa, n, d_max));
            uint32_t hmax[LH_MAX_LEVELS] = {0};
            STEP(lh_readback(ctx, d_max, L * sizeof(uint32_t), hmax));
            for (uint32_t l = 0; l < L; ++l) bits[l] = hmax[l] ? 32 - __builtin_clz(hmax[l]) : 1;
        }
    }
    for (uint32_t l = 0; l < L; ++l) {
        t->key_bits[l] = bits[l];
        total_bits += bits[l];
    }
    if (s == LH_OK && total_bits > 64)
        s = lh_fail(ctx, LH_EUNSUPPORTED, "packed key needs %u > 64 bits", total_bits);
    // 2. pack + sort
    uint32_t shift[LH_MAX_LEVELS];
    {
        uint32_t acc = 0;
        for (int l = (int)L - 1; l >= 0; --l) {  // level 0 most significant
            shift[l] = acc;
            acc += bits[l];
        }
        for (uint32_t l = 0; l < L; ++l) pa.shift[l] = shift[l];
    }
    // one 4-byte FIRST / f32 SUM annotation is sorted along with the keys
    // instead of the row ids, so leaf order needs no gather through them
    const bool carry = rel->nannos == 1 && dtype_size(rel->anno_types[0]) == 4 &&
                       (merge == LH_MERGE_FIRST || (merge == LH_MERGE_SUM && rel->anno_types[0] == LH_T_F32));
    pa.payload = carry ? (const uint32_t *)rel->annos[0] : nullptr;
    STEP(lh_alloc(ctx, &key, n));
    STEP(lh_alloc(ctx, &tkey, n));
    STEP(lh_alloc(ctx, &rid, n));
    STEP(lh_alloc(ctx, &trid, n));
    // one readback block: level counts, the status word (key bounds, sort and
    // level waits), then the layout totals (bitset sets, words) per level
    const size_t n_rb = L + 1 + 2 * LH_MAX_LEVELS;
    STEP(lh_alloc(ctx, &d_count, n_rb));
    if (s == LH_OK) {
        cudaError_t e = cudaMemsetAsync(d_count, 0, n_rb * sizeof(uint64_t), ctx->stream);
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "build_trie: %s", cudaGetErrorString(e));
    }
    pa.status = d_count ? (uint32_t *)(d_count + L) : nullptr;
    pa.passes = (int)((total_bits + 7) / 8);
    STEP(lh_alloc(ctx, &d_hist, (size_t)8 * 256));
    if (s == LH_OK) {
        cudaError_t e = cudaMemsetAsync(d_hist, 0, (size_t)8 * 256 * sizeof(unsigned long long), ctx->stream);
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "build_trie: %s", cudaGetErrorString(e));
    }
    pa.hist = d_hist;
    if (s == LH_OK && n) {
        LH_TRACED(ctx, "k_pack", k_pack<<<G4, T, 0, ctx->stream>>>(pa, n, key, rid));
        STEP(lh_radix_sort_u64(ctx, &key, &rid, &tkey, &trid, n, (int)total_bits, (uint32_t *)(d_count + L), d_hist));
    }
    // 3. levels: the leaf level is written in place (capacity n), the levels
    //    above into temporaries, copied out once their sizes are known
    const uint64_t lvt = lv_tile((int)L);
    const uint64_t ntiles = (n + lvt - 1) / lvt;
    STEP(trie_alloc(ctx, t, &t->lv[L - 1].vals, n));
    STEP(lh_alloc(ctx, &runstart, n));
    STEP(lh_alloc(ctx, &ticket, 1));
    STEP(lh_alloc(ctx, &lstate, ntiles * L));
    for (uint32_t l = 0; l + 1 < L; ++l) {
        STEP(lh_alloc(ctx, &tvals[l], n));
        STEP(lh_alloc(ctx, &toffs[l], n + 1));
    }
    uint64_t cnt[3 * LH_MAX_LEVELS + 1] = {0};
    if (s == LH_OK && n) {
        if (ntiles >= (1ull << 32)) s = lh_fail(ctx, LH_EOVERFLOW, "too many level tiles");
        LevelArgs la;
        memset(&la, 0, sizeof(la));
        la.nlev = L;
        for (uint32_t l = 0; l < L; ++l) {
            la.shift[l] = shift[l];
            la.vmask[l] = bits[l] >= 32 ? 0xFFFFFFFFu : ((1u << bits[l]) - 1u);
            la.vals[l] = l + 1 < L ? tvals[l] : t->lv[l].vals;
            la.offs[l] = l + 1 < L ? toffs[l] : nullptr;
        }
        la.runstart = runstart;
        la.state = lstate;
        la.ticket = ticket;
        la.count = d_count;
        la.status = (uint32_t *)(d_count + L);
        if (s == LH_OK) {
            cudaMemsetAsync(lstate, 0, ntiles * L * sizeof(unsigned long long), ctx->stream);
            cudaMemsetAsync(ticket, 0, sizeof(uint32_t), ctx->stream);
            const unsigned nt = (unsigned)ntiles;
            switch (L) {
                case 1: LH_TRACED(ctx, "k_levels", k_levels<1><<<nt, kLvThreads, 0, ctx->stream>>>(key, n, la)); break;
                case 2: LH_TRACED(ctx, "k_levels", k_levels<2><<<nt, kLvThreads, 0, ctx->stream>>>(key, n, la)); break;
                case 3: LH_TRACED(ctx, "k_levels", k_levels<3><<<nt, kLvThreads, 0, ctx->stream>>>(key, n, la)); break;
                case 4: LH_TRACED(ctx, "k_levels", k_levels<4><<<nt, kLvThreads, 0, ctx->stream>>>(key, n, la)); break;
                case 5: LH_TRACED(ctx, "k_levels", k_levels<5><<<nt, kLvThreads, 0, ctx->stream>>>(key, n, la)); break;
                default: LH_TRACED(ctx, "k_levels", k_levels<6><<<nt, kLvThreads, 0, ctx->stream>>>(key, n, la)); break;
            }
        }
        // layout decisions on the level arrays as written (upper levels still
        // in their temporaries), set counts read on the device
        if (s == LH_OK && any_ratio) {
            unsigned long long *d_tot = (unsigned long long *)(d_count + L + 1);
            for (uint32_t l = 0; l < L && s == LH_OK; ++l) {
                const uint64_t cap_sets = l ? n : 1;
                STEP(lh_alloc(ctx, &pre.isbs[l], cap_sets));
                STEP(lh_alloc(ctx, &pre.words[l], cap_sets));
                if (s != LH_OK) break;
                const uint32_t *lv_vals = l + 1 < L ? tvals[l] : t->lv[l].vals;
                const uint32_t *poffs = l ? toffs[l - 1] : nullptr;
                LH_TRACED(ctx, "k_layout_decide", k_layout_decide<<<lh_blocks(cap_sets, T, (uint32_t)ctx->num_sms * 16), T, 0, ctx->stream>>>(
                    lv_vals, poffs, 1, 0, l ? d_count + (l - 1) : nullptr, d_count + l, t->level_ratio[l],
                    pol.bs_min_card, pre.isbs[l], pre.words[l], d_tot + 2 * l));
            }
        }
        STEP(lh_readback(ctx, d_count, n_rb * sizeof(uint64_t), cnt));
        if (s == LH_OK) memcpy(pre.tot, cnt + L + 1, sizeof(pre.tot));
        if (s == LH_OK && (uint32_t)cnt[L])
            s = lh_fail(ctx, (lh_status)(uint32_t)cnt[L], (uint32_t)cnt[L] == LH_EINVAL
                                                              ? "build_trie: a key value is at or above its key_bound"
                                                              : "build_trie: a bounded wait (sort or level offsets) gave up");
    }
    for (uint32_t l = 0; l < L; ++l) t->lv[l].n = cnt[l];
    nu = cnt[L - 1];
    for (uint32_t l = 0; l + 1 < L && s == LH_OK; ++l) {
        TrieLevel &lv = t->lv[l];
        STEP(trie_alloc(ctx, t, &lv.vals, lv.n));
        STEP(trie_alloc(ctx, t, &lv.offs, lv.n + 1));
        if (s == LH_OK && lv.n) {
            cudaError_t e = cudaMemcpyAsync(lv.vals, tvals[l], lv.n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(lv.offs, toffs[l], (lv.n + 1) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctx->stream);
            if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "build_trie copy: %s", cudaGetErrorString(e));
        } else if (s == LH_OK) {
            cudaError_t e = cudaMemsetAsync(lv.offs, 0, sizeof(uint32_t), ctx->stream);
            if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "build_trie: %s", cudaGetErrorString(e));
        }
    }
    // 4. annotations in leaf order
    if (s == LH_OK && carry) {
        t->nannos = 1;
        t->anno_type[0] = rel->anno_types[0];
        if (nu == n) {
            // no duplicates: the sorted payload is the leaf-order column
            t->anno[0] = rid;
            t->allocs.push_back((void *)rid);
            t->bytes += (n ? n : 1) * sizeof(uint32_t);
            rid = nullptr;
        } else {
            uint32_t *p = nullptr;
            STEP(trie_alloc(ctx, t, &p, nu));
            t->anno[0] = p;
            if (s == LH_OK && nu)
                LH_TRACED(ctx, "k_annos_carried", k_annos_carried<<<G, T, 0, ctx->stream>>>(
                                                      rid, runstart, nu, n, merge == LH_MERGE_SUM ? 1u : 0u, p));
        }
    } else if (s == LH_OK && rel->nannos) {
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
    if (s == LH_OK && n && any_ratio) s = trie_layout(ctx, t, &pre);
    else STEP(lh_trie_layout(ctx, t));
    free_pre();
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
    t->level_ratio[0] = pol.per_level ? pol.level_ratio[0] : pol.bs_ratio;
    const unsigned T = 256;
    const unsigned G = (unsigned)std::min<uint64_t>(lh_blocks(n, T), (uint64_t)ctx->num_sms * 16);
    const unsigned G4 = (unsigned)std::min<uint64_t>(lh_blocks((n + 3) / 4, T), (uint64_t)ctx->num_sms * 16);
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

// ------------------------------------------------ selection pushed into a build

namespace {
__global__ void k_where_flags(lh_row_filter f0, lh_row_filter f1, lh_row_filter f2, lh_row_filter f3, uint32_t nf,
                              uint64_t n, uint32_t *flag) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        bool ok = true;
        const lh_row_filter fs[4] = {f0, f1, f2, f3};
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k)
            if (k < nf) {
                const int32_t v = fs[k].col[i];
                ok = ok && v >= fs[k].lo && v <= fs[k].hi;
            }
        flag[i] = ok ? 1u : 0u;
    }
}

template <class T>
__global__ void k_where_gather(const T *src, const uint32_t *flag, const uint32_t *pos, uint64_t n, T *dst) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (flag[i]) dst[pos[i]] = src[i];
}

template <class T>
lh_status where_gather(lh_ctx *ctx, const void *src, const uint32_t *flag, const uint32_t *pos, uint64_t n,
                       uint64_t cnt, void **dst) {
    T *d = nullptr;
    LH_TRY(lh_alloc(ctx, &d, std::max<uint64_t>(cnt, 1)));
    const unsigned G = (unsigned)std::min<uint64_t>(lh_blocks(n, 256), (uint64_t)ctx->num_sms * 16);
    if (n) LH_TRACED(ctx, "k_where_gather", k_where_gather<T><<<G, 256, 0, ctx->stream>>>((const T *)src, flag, pos, n, d));
    *dst = d;
    return LH_OK;
}
}  // namespace

extern "C" lh_status lh_build_trie_where(lh_ctx *ctx, const lh_relation_desc *rel, const uint32_t *key_order,
                                         const lh_layout_policy *layout, lh_merge merge, const lh_row_filter *where,
                                         uint32_t n_where, lh_trie **out) {
    if (!ctx || !rel || !out) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (n_where > 4 || (n_where && !where)) return lh_fail(ctx, LH_EINVAL, "0..4 row filters");
    for (uint32_t k = 0; k < n_where; ++k)
        if (!where[k].col && rel->nrows) return lh_fail(ctx, LH_EINVAL, "row filter %u: null column", k);
    if (rel->nkeys == 0 || rel->nkeys > LH_MAX_LEVELS || rel->nannos > LH_MAX_ANNOS)
        return lh_fail(ctx, LH_EINVAL, "bad relation shape");
    if (n_where == 0) return lh_build_trie(ctx, rel, key_order, layout, merge, out);
    const uint64_t n = rel->nrows;
    if (n >= (1ull << 32)) return lh_fail(ctx, LH_EOVERFLOW, "more than 2^32-1 rows");
    lh_row_filter f[4] = {};
    for (uint32_t k = 0; k < n_where; ++k) f[k] = where[k];
    for (uint32_t k = n_where; k < 4; ++k) f[k] = f[0];
    uint32_t *flag = nullptr, *pos = nullptr;
    lh_status s = lh_alloc(ctx, &flag, std::max<uint64_t>(n, 1));
    if (s == LH_OK) s = lh_alloc(ctx, &pos, n + 1);
    const unsigned G = (unsigned)std::min<uint64_t>(lh_blocks(n, 256), (uint64_t)ctx->num_sms * 16);
    if (s == LH_OK && n) LH_TRACED(ctx, "k_where_flags", k_where_flags<<<G, 256, 0, ctx->stream>>>(f[0], f[1], f[2], f[3], n_where, n, flag));
    if (s == LH_OK) s = lh_scan_u32_to_u32(ctx, flag, pos, n);
    uint32_t cnt = 0;
    if (s == LH_OK) s = lh_readback(ctx, pos + n, sizeof(uint32_t), &cnt);
    // the selected rows as a relation of their own, then the ordinary build
    lh_relation_desc sel = *rel;
    sel.nrows = cnt;
    std::vector<void *> temps;
    for (uint32_t c = 0; c < rel->nkeys && s == LH_OK; ++c) {
        void *d = nullptr;
        s = where_gather<uint32_t>(ctx, rel->keys[c], flag, pos, n, cnt, &d);
        temps.push_back(d);
        sel.keys[c] = (const uint32_t *)d;
    }
    for (uint32_t c = 0; c < rel->nannos && s == LH_OK; ++c) {
        void *d = nullptr;
        switch (rel->anno_types[c]) {
            case LH_T_F64: s = where_gather<uint64_t>(ctx, rel->annos[c], flag, pos, n, cnt, &d); break;
            case LH_T_I8: s = where_gather<uint8_t>(ctx, rel->annos[c], flag, pos, n, cnt, &d); break;
            default: s = where_gather<uint32_t>(ctx, rel->annos[c], flag, pos, n, cnt, &d); break;
        }
        temps.push_back(d);
        sel.annos[c] = d;
    }
    if (s == LH_OK) s = lh_build_trie(ctx, &sel, key_order, layout, merge, out);
    lh_free(ctx, flag);
    lh_free(ctx, pos);
    for (void *p : temps) lh_free(ctx, p);
    return s;
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
