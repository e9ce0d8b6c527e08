// Sparse linear algebra as join-aggregates.
//
// SpMV  y(i) = sum_j A(i,j) x(j): x is a completely dense relation, so the
//   j attribute needs no intersection (Section 4.1.1, icost 0); every row of
//   A's trie is reduced by a 16-lane group with fp32 error-free products and
//   compensated sums.
// SpGEMM C(i,k) = sum_j A(i,j) B(j,k) in the order [i, j, k] with j projected
//   away before the materialised k (Section 4.1.2 relaxation): per row i,
//   j ranges over A(i) cap pi_j B (a probe of B's first level), and the k
//   values of every B(j) are unioned with a GROUP BY on the key k (Section 5)
//   whose accumulator is a hash table (keys + compensated fp32 value pairs)
//   in shared memory, or in global memory for rows whose bound exceeds it.
//   Each row's result is sorted (bitonic) so C's rows are sorted sets.
#include "lh_join.cuh"

namespace {

// ------------------------------------------------------------------ SpMV

constexpr int kSpmvThreads = 256;
constexpr int kSpmvGroup = 16;

// Each 16-lane group handles kSpmvRows rows per iteration (rows g, g + G,
// ...), so their offset loads, first element loads and x gathers are all in
// flight together; rows longer than 16 entries finish in a loop.
constexpr int kSpmvRows = 4;

__global__ void __launch_bounds__(kSpmvThreads) k_spmv(DTrie A, const float *av, const float *x,
                                                       uint32_t x_n, uint32_t nrow_entries, float *y) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & (kSpmvGroup - 1);
    const uint32_t group = (blockIdx.x * blockDim.x + threadIdx.x) / kSpmvGroup;
    const uint32_t ngroups = (gridDim.x * blockDim.x) / kSpmvGroup;
    const uint32_t *rows = A.lv[0].vals, *offs = A.lv[0].offs, *cols = A.lv[1].vals;
    const uint64_t stride = (uint64_t)ngroups * kSpmvRows;
    for (uint64_t p0 = group - (group % 2); p0 < nrow_entries; p0 += stride) {
        // both half-warps iterate together so the shuffles stay converged
        uint32_t lo[kSpmvRows], hi[kSpmvRows];
        bool valid[kSpmvRows];
#pragma unroll
        for (int u = 0; u < kSpmvRows; ++u) {
            const uint64_t p = p0 + (group % 2) + (uint64_t)u * ngroups;
            valid[u] = p < nrow_entries;
            lo[u] = valid[u] ? __ldg(offs + p) : 0u;
            hi[u] = valid[u] ? __ldg(offs + p + 1) : 0u;
        }
        uint32_t j[kSpmvRows];
        float a[kSpmvRows], xv[kSpmvRows];
#pragma unroll
        for (int u = 0; u < kSpmvRows; ++u) {
            const uint32_t q = lo[u] + sub;
            const bool in = q < hi[u];
            j[u] = in ? __ldg(cols + q) : 0xFFFFFFFFu;
            a[u] = in ? __ldg(av + q) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kSpmvRows; ++u) xv[u] = j[u] < x_n ? __ldg(x + j[u]) : 0.f;  // x holds keys [0, x_n)
        float sh[kSpmvRows], sl[kSpmvRows];
#pragma unroll
        for (int u = 0; u < kSpmvRows; ++u) {
            sh[u] = 0.f;
            sl[u] = 0.f;
            if (j[u] < x_n) {
                float ph, pl;
                lh_two_prod(a[u], xv[u], ph, pl);
                lh_pair_add(sh[u], sl[u], ph, pl);
            }
            for (uint32_t q = lo[u] + sub + kSpmvGroup; q < hi[u]; q += kSpmvGroup) {
                const uint32_t jj = __ldg(cols + q);
                if (jj >= x_n) continue;
                float ph, pl;
                lh_two_prod(__ldg(av + q), __ldg(x + jj), ph, pl);
                lh_pair_add(sh[u], sl[u], ph, pl);
            }
        }
#pragma unroll
        for (int u = 0; u < kSpmvRows; ++u) {
#pragma unroll
            for (int o = kSpmvGroup / 2; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(LH_FULL, sh[u], o), ol = __shfl_xor_sync(LH_FULL, sl[u], o);
                lh_pair_add(sh[u], sl[u], oh, ol);
            }
            if (valid[u] && sub == 0) y[__ldg(rows + p0 + (group % 2) + (uint64_t)u * ngroups)] = sh[u] + sl[u];
        }
    }
}

// ---------------------------------------------------------------- SpGEMM

constexpr int kGemmWarps = 4;
constexpr int kGemmThreads = kGemmWarps * 32;
constexpr uint32_t kTab = 512;      // shared hash slots per warp
constexpr uint32_t kSortMax = 256;  // entries sortable in shared memory per warp
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t hash_k(uint32_t k) { return k * 2654435761u; }

// Upper bound of |C(i,.)| per row entry p of A: sum of |B(j)| over j in A(i)
// that B has.
__global__ void k_spgemm_bound(DTrie A, DTrie B, uint32_t nA0, uint32_t *ub) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nA0; p += gridDim.x * blockDim.x) {
        const uint32_t lo = __ldg(A.lv[0].offs + p), hi = __ldg(A.lv[0].offs + p + 1);
        uint64_t u = 0;
        for (uint32_t q = lo; q < hi; ++q) {
            uint32_t pj;
            if (lh_probe(B, 0, 0, 0, B.lv[0].n, __ldg(A.lv[1].vals + q), &pj))
                u += __ldg(B.lv[0].offs + pj + 1) - __ldg(B.lv[0].offs + pj);
        }
        ub[p] = (uint32_t)(u < 0xFFFFFFFFull ? u : 0xFFFFFFFFull);
    }
}

// Global hash capacity for rows above the shared bound (0 for the others),
// and the number of rows the sort-based kernel does not take (more than
// 256 products or more than 32 A entries).
// sizes[0..1] = (U, hash rows); the hash-row counter is sizes[0] on entry
__global__ void k_spgemm_sizes(const uint64_t *u_end, unsigned long long *sizes) {
    if (threadIdx.x == 0) {
        const unsigned long long h = sizes[0];
        sizes[0] = *u_end;
        sizes[1] = h;
    }
}

// ---- GROUP BY key: hash or bitset + dense array (Section 5) -----------------
// The union over j of the rows B(j) is a GROUP BY on the key k.  A row whose
// possible outputs span at most kDenseSpan values, and which is predicted to
// fill its span densely (at least one product per kDenseRatio values of the
// span), unions its keys as bits and sums its values in a dense array; the
// other rows sort (<= 256 products) or hash.  dense_mode 0: never dense, 1:
// the density rule for rows the sort path does not take, 2: every row whose
// span fits.
constexpr uint32_t kDenseSpan = 4096;
constexpr uint32_t kDenseRatio = 4;
enum { ROW_SORT = 0, ROW_HASH = 1, ROW_DENSE = 2 };

__global__ void k_spgemm_gcap(DTrie A, DTrie B, const uint32_t *ub, uint32_t n, uint32_t dense_mode, uint64_t *gcap,
                              uint8_t *kind, uint32_t *kmin, unsigned long long *n_rows) {
    unsigned long long mine = 0, dense = 0;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint64_t u = ub[p];
        const uint32_t alo = __ldg(A.lv[0].offs + p), ahi = __ldg(A.lv[0].offs + p + 1);
        const bool sortable = u <= kTab / 2 && ahi - alo <= 32;  // the sort path's rows (kEscPairs)
        uint32_t kd = sortable ? ROW_SORT : ROW_HASH;
        uint32_t lo_k = 0;
        if (u > 0 && (dense_mode == 2 || (dense_mode == 1 && !sortable))) {
            // span of the row's possible outputs: first and last k of every B(j)
            uint32_t mn = 0xFFFFFFFFu, mx = 0;
            for (uint32_t q = alo; q < ahi; ++q) {
                uint32_t pj;
                if (!lh_probe(B, 0, 0, 0, B.lv[0].n, __ldg(A.lv[1].vals + q), &pj)) continue;
                const uint32_t b0 = __ldg(B.lv[0].offs + pj), b1 = __ldg(B.lv[0].offs + pj + 1);
                if (b1 == b0) continue;
                mn = min(mn, __ldg(B.lv[1].vals + b0));
                mx = max(mx, __ldg(B.lv[1].vals + b1 - 1));
            }
            if (mx >= mn) {
                const uint64_t span = (uint64_t)mx - mn + 1;
                if (span <= kDenseSpan && (dense_mode == 2 || u * kDenseRatio >= span)) {
                    kd = ROW_DENSE;
                    lo_k = mn;
                }
            }
        }
        uint64_t c = 0;
        if (kd == ROW_HASH && u > kTab / 2) {
            c = 64;
            while (c < 2 * u) c <<= 1;
        }
        gcap[p] = c;
        kind[p] = (uint8_t)kd;
        kmin[p] = lo_k;
        // rows for the hash kernel: the non-sortable ones, and with
        // dense_mode 2 (no sort kernel) the sortable ones too
        mine += (kd == ROW_HASH || (dense_mode == 2 && kd == ROW_SORT)) ? 1ull : 0ull;
        dense += kd == ROW_DENSE ? 1ull : 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mine += __shfl_xor_sync(LH_FULL, mine, o);
        dense += __shfl_xor_sync(LH_FULL, dense, o);
    }
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(n_rows, mine);
    if ((threadIdx.x & 31) == 0 && dense) atomicAdd(n_rows + 2, dense);
}

constexpr int kDenseThreads = 256;

struct DenseSmem {
    double acc[kDenseSpan];
    uint32_t bits[kDenseSpan / 32];
    uint32_t wpre[kDenseSpan / 32];
    uint32_t jb[kDenseThreads], jl[kDenseThreads], jp[kDenseThreads];
    float ja[kDenseThreads];
    uint32_t warp_tot[kDenseThreads / 32];
};

// inclusive block scan of one value per thread (256 threads)
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t *warp_tot) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(LH_FULL, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    uint32_t add = 0;
    for (uint32_t w = 0; w < warp; ++w) add += warp_tot[w];
    __syncthreads();
    return x + add;
}

// One block per dense row: every product adds its exact fp64 value a * b to
// its key's slot and sets the key's bit; the set bits, in ascending order,
// then give the row's result already sorted (no sort, no hash).  The fp64
// slots are the row's final per-key totals.
__global__ void __launch_bounds__(kDenseThreads) k_spgemm_dense(
    DTrie A, const float *av, DTrie B, const float *bv, uint32_t nA0, const uint8_t *kind, const uint32_t *kmin,
    const uint64_t *tmp_off, uint32_t *tcol, float *tval, uint32_t *cnt) {
    extern __shared__ __align__(16) unsigned char dn_raw[];
    DenseSmem &S = *(DenseSmem *)dn_raw;
    const uint32_t tid = threadIdx.x;
    for (uint32_t p = blockIdx.x; p < nA0; p += gridDim.x) {
        if (kind[p] != ROW_DENSE) continue;
        const uint32_t k0 = kmin[p];
        for (uint32_t i = tid; i < kDenseSpan; i += kDenseThreads) S.acc[i] = 0.0;
        for (uint32_t i = tid; i < kDenseSpan / 32; i += kDenseThreads) S.bits[i] = 0u;
        __syncthreads();
        const uint32_t alo = __ldg(A.lv[0].offs + p), ahi = __ldg(A.lv[0].offs + p + 1);
        for (uint32_t q0 = alo; q0 < ahi; q0 += kDenseThreads) {
            const uint32_t q = q0 + tid;
            uint32_t bstart = 0, blen = 0;
            float a = 0.f;
            if (q < ahi) {
                uint32_t pj;
                if (lh_probe(B, 0, 0, 0, B.lv[0].n, __ldg(A.lv[1].vals + q), &pj)) {
                    bstart = __ldg(B.lv[0].offs + pj);
                    blen = __ldg(B.lv[0].offs + pj + 1) - bstart;
                    a = __ldg(av + q);
                }
            }
            const uint32_t incl = block_incl_scan(blen, S.warp_tot);
            S.jb[tid] = bstart;
            S.jl[tid] = blen;
            S.jp[tid] = incl;
            S.ja[tid] = a;
            __syncthreads();
            const uint32_t total = S.jp[kDenseThreads - 1];
            for (uint32_t t = tid; t < total; t += kDenseThreads) {
                uint32_t lo = 0, hi = kDenseThreads - 1;  // first staged entry with prefix > t
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (S.jp[mid] > t) hi = mid;
                    else lo = mid + 1;
                }
                const uint32_t pos = S.jb[lo] + (t - (S.jp[lo] - S.jl[lo]));
                const uint32_t d = __ldg(B.lv[1].vals + pos) - k0;
                atomicAdd(&S.acc[d], (double)S.ja[lo] * (double)__ldg(bv + pos));   // exact product in fp64
                atomicOr(&S.bits[d >> 5], 1u << (d & 31u));
            }
            __syncthreads();
        }
        // compaction in key order
        const uint32_t w = tid;  // kDenseSpan / 32 == 128 words, one per thread below 128
        const uint32_t c = w < kDenseSpan / 32 ? __popc(S.bits[w]) : 0u;
        const uint32_t incl = block_incl_scan(c, S.warp_tot);
        const uint64_t t0 = tmp_off[p];
        if (w < kDenseSpan / 32) {
            uint32_t bitsw = S.bits[w], o = incl - c;
            while (bitsw) {
                const uint32_t b = __ffs(bitsw) - 1;
                bitsw &= bitsw - 1;
                tcol[t0 + o] = k0 + 32 * w + b;
                tval[t0 + o] = (float)S.acc[32 * w + b];
                ++o;
            }
        }
        if (tid == kDenseThreads - 1) cnt[p] = incl;
        __syncthreads();
    }
}

struct WarpSmem {
    uint32_t key[kTab];
    float hi[kTab];
    float lo[kTab];
    uint32_t skey[kSortMax];
    float sval[kSortMax];
    float st_h[32], st_l[32];
    uint32_t jb[32], jl[32], jp[32];  // B row start, length, inclusive prefix of lengths
    float ja[32];                      // A(i,j) value
};

// (key, value) pairs in [0, n) of warp-visible memory sorted ascending by key
// (bitonic network over the next power of two, padding keys = kEmpty).
__device__ void warp_bitonic(uint32_t *key, float *val, uint32_t n, uint32_t npow) {
    const int lane = threadIdx.x & 31;
    for (uint32_t t = n + lane; t < npow; t += 32) key[t] = kEmpty;
    __syncwarp();
    for (uint32_t k = 2; k <= npow; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t t = lane; t < npow; t += 32) {
                const uint32_t u = t ^ j;
                if (u > t) {
                    const bool up = (t & k) == 0;
                    const uint32_t a = key[t], b = key[u];
                    if ((a > b) == up) {
                        key[t] = b;
                        key[u] = a;
                        const float va = val[t];
                        val[t] = val[u];
                        val[u] = va;
                    }
                }
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(kGemmThreads) k_spgemm_numeric(
    DTrie A, const float *av, DTrie B, const float *bv, uint32_t nA0, const uint64_t *tmp_off,
    const uint64_t *goff, uint32_t *gkey, float *ghi, float *glo, uint32_t *tcol, float *tval,
    uint32_t *cnt, const uint8_t *kind, uint32_t take_sort_rows) {
    __shared__ WarpSmem sm_all[kGemmWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem &S = sm_all[warp];
    const uint32_t gw = blockIdx.x * kGemmWarps + warp;
    const uint32_t nw = gridDim.x * kGemmWarps;
    for (uint32_t p = gw; p < nA0; p += nw) {
        const uint64_t cap64 = goff[p + 1] - goff[p];
        const bool global = cap64 > 0;
        // dense rows have their own kernel; sortable rows go to k_spgemm_esc
        // unless no sort kernel runs
        const uint8_t kd = kind[p];
        if (kd == ROW_DENSE || (kd == ROW_SORT && !take_sort_rows)) continue;
        const uint32_t cap = global ? (uint32_t)cap64 : kTab;
        uint32_t *key = global ? gkey + goff[p] : S.key;
        float *th = global ? ghi + goff[p] : S.hi;
        float *tl = global ? glo + goff[p] : S.lo;
        for (uint32_t s = lane; s < cap; s += 32) {
            key[s] = kEmpty;
            th[s] = 0.f;
            tl[s] = 0.f;
        }
        __syncwarp();
        const uint32_t alo = __ldg(A.lv[0].offs + p), ahi = __ldg(A.lv[0].offs + p + 1);
        for (uint32_t q0 = alo; q0 < ahi; q0 += 32) {
            // stage up to 32 (j, a) of this row with their B row ranges
            const uint32_t q = q0 + lane;
            uint32_t bstart = 0, blen = 0;
            float a = 0.f;
            if (q < ahi) {
                uint32_t pj;
                if (lh_probe(B, 0, 0, 0, B.lv[0].n, __ldg(A.lv[1].vals + q), &pj)) {
                    bstart = __ldg(B.lv[0].offs + pj);
                    blen = __ldg(B.lv[0].offs + pj + 1) - bstart;
                    a = __ldg(av + q);
                }
            }
            uint32_t incl = blen;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(LH_FULL, incl, o);
                if (lane >= o) incl += t;
            }
            S.jb[lane] = bstart;
            S.jl[lane] = blen;
            S.jp[lane] = incl;
            S.ja[lane] = a;
            const uint32_t total = __shfl_sync(LH_FULL, incl, 31);
            __syncwarp();
            for (uint32_t t0 = 0; t0 < total; t0 += 32) {
                const uint32_t t = t0 + lane;
                const bool act = t < total;
                uint32_t k = kEmpty;
                float ph = 0.f, pl = 0.f;
                if (act) {
                    uint32_t lo = 0, hi = 31;  // first staged j with prefix > t
                    while (lo < hi) {
                        uint32_t mid = (lo + hi) >> 1;
                        if (S.jp[mid] > t) hi = mid;
                        else lo = mid + 1;
                    }
                    const uint32_t pos = S.jb[lo] + (t - (S.jp[lo] - S.jl[lo]));
                    k = __ldg(B.lv[1].vals + pos);
                    lh_two_prod(S.ja[lo], __ldg(bv + pos), ph, pl);
                }
                // lanes that share a k merge their terms first, then one lane updates
                const uint32_t peers = __match_any_sync(LH_FULL, k);
                S.st_h[lane] = ph;
                S.st_l[lane] = pl;
                __syncwarp();
                if (act && (peers & ((1u << lane) - 1u)) == 0) {
                    float sh = 0.f, sl = 0.f;
                    uint32_t m = peers;
                    while (m) {
                        const int s = __ffs(m) - 1;
                        m &= m - 1;
                        lh_pair_add(sh, sl, S.st_h[s], S.st_l[s]);
                    }
                    uint32_t slot = hash_k(k) & (cap - 1);
                    for (uint32_t probe = 0; probe < cap; ++probe) {
                        const uint32_t prev = atomicCAS(&key[slot], kEmpty, k);
                        if (prev == kEmpty || prev == k) break;
                        slot = (slot + 1) & (cap - 1);
                    }
                    float ch = th[slot], cl = tl[slot];
                    lh_pair_add(ch, cl, sh, sl);
                    th[slot] = ch;
                    tl[slot] = cl;
                }
                __syncwarp();
            }
        }
        // compact occupied slots, sort by k, write the row to its temporary range
        uint32_t n = 0;
        uint32_t *ok_ = global ? gkey + goff[p] : S.skey;  // compaction target
        float *ov = global ? ghi + goff[p] : S.sval;
        if (!global) {
            for (uint32_t s0 = 0; s0 < cap; s0 += 32) {
                const uint32_t s = s0 + lane;
                const bool occ = s < cap && key[s] != kEmpty;
                const uint32_t b = __ballot_sync(LH_FULL, occ);
                if (occ) {
                    const uint32_t d = n + __popc(b & ((1u << lane) - 1u));
                    ok_[d] = key[s];
                    ov[d] = th[s] + tl[s];
                }
                n += __popc(b);
            }
        } else {
            // in place: compacted index never passes the slot it reads
            for (uint32_t s0 = 0; s0 < cap; s0 += 32) {
                const uint32_t s = s0 + lane;
                const bool occ = s < cap && key[s] != kEmpty;
                const uint32_t kk = occ ? key[s] : 0u;
                const float vv = occ ? th[s] + tl[s] : 0.f;
                const uint32_t b = __ballot_sync(LH_FULL, occ);
                __syncwarp();
                if (occ) {
                    const uint32_t d = n + __popc(b & ((1u << lane) - 1u));
                    ok_[d] = kk;
                    ov[d] = vv;
                }
                n += __popc(b);
                __syncwarp();
            }
        }
        __syncwarp();
        uint32_t npow = 1;
        while (npow < n) npow <<= 1;
        if (n > 1) warp_bitonic(ok_, ov, n, npow);
        const uint64_t t0 = tmp_off[p];
        for (uint32_t s = lane; s < n; s += 32) {
            tcol[t0 + s] = ok_[s];
            tval[t0 + s] = ov[s];
        }
        if (lane == 0) cnt[p] = n;
        __syncwarp();
    }
}

// ---- sort-based rows (expand, sort, compress) -------------------------------
// A row with at most kEscPairs products: lane L expands products 8L..8L+7 of
// the concatenated B rows into registers as 64-bit keys (k << 8 | product
// index); a bitonic network over the 256 positions p = 8 * lane + e sorts
// them (register compare-exchanges for distances < 8, shuffles for larger
// ones); equal k are then adjacent.  Runs are summed in registers with
// compensated fp32 arithmetic: each lane sums its 8 positions, and a
// segmented suffix scan over lanes carries a run across lane boundaries.
// Each run is written once, already in ascending k.
constexpr uint32_t kEscPairs = 256;
constexpr int kEscWarps = 8;

struct EscSmem {
    float2 val[kEscPairs];
    uint32_t jb[32], jl[32], jp[32];
    float ja[32];
};

// Bitonic network over 256 keys held 8 per lane at positions p = 8 * lane + e,
// fully unrolled so every distance and direction test is a constant:
// distances below 8 are register compare-exchanges, larger ones shuffles.
// FIRST: first merge stage (log2 of the run length it produces); runs of
// length 2^(FIRST-1) must already be sorted, ascending for even run index
// and descending for odd.
template <class K, int FIRST = 1>
__device__ __forceinline__ void esc_sort256(K (&key)[8], uint32_t lane) {
#pragma unroll
    for (int kk = FIRST; kk <= 8; ++kk) {
        const uint32_t k = 1u << kk;
#pragma unroll
        for (int jj = kk - 1; jj >= 0; --jj) {
            const uint32_t j = 1u << jj;
            if (j >= 8) {
                const uint32_t lj = j >> 3;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const bool up = k >= 8 ? ((lane & (k >> 3)) == 0) : ((e & k) == 0);
                    const K other = __shfl_xor_sync(LH_FULL, key[e], lj);
                    const K mn = key[e] < other ? key[e] : other;
                    const K mx = key[e] < other ? other : key[e];
                    key[e] = (lower == up) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if ((e & j) == 0) {
                        const bool up = k >= 8 ? ((lane & (k >> 3)) == 0) : ((e & k) == 0);
                        const K x = key[e], y = key[e + j];
                        const K mn = x < y ? x : y, mx = x < y ? y : x;
                        key[e] = up ? mn : mx;
                        key[e + j] = up ? mx : mn;
                    }
                }
            }
        }
    }
}

// shared slot of product t = 8 * lane + e: lane-major, so the expand
// phase's stores of one e hit 32 consecutive float2
__device__ __forceinline__ uint32_t esc_vslot(uint32_t t) { return ((t & 7u) << 5) | (t >> 3); }

// K = uint32_t when every k < 2^24 (k << 8 | index fits 32 bits), else uint64_t.
// One row of the sort-based path: the row's results, ascending in k, go to
// ocol / oval (global or shared memory); returns their count (all lanes).
template <class K>
__device__ __forceinline__ uint32_t esc_row(const DTrie &A, const float *av, const DTrie &B, const float *bv,
                                            uint32_t p, EscSmem &S, uint32_t lane, uint32_t *ocol, float *oval) {
        const uint32_t alo = __ldg(A.lv[0].offs + p), ahi = __ldg(A.lv[0].offs + p + 1);
        // stage the row's (j, a) with their B row ranges
        const uint32_t q = alo + lane;
        uint32_t bstart = 0, blen = 0;
        float a = 0.f;
        if (q < ahi) {
            uint32_t pj;
            if (lh_probe(B, 0, 0, 0, B.lv[0].n, __ldg(A.lv[1].vals + q), &pj)) {
                bstart = __ldg(B.lv[0].offs + pj);
                blen = __ldg(B.lv[0].offs + pj + 1) - bstart;
                a = __ldg(av + q);
            }
        }
        uint32_t incl = blen;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(LH_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        S.jb[lane] = bstart;
        S.jl[lane] = blen;
        S.jp[lane] = incl;
        S.ja[lane] = a;
        const uint32_t total = __shfl_sync(LH_FULL, incl, 31);
        __syncwarp();
        // rows whose B rows all have one power-of-two length L (4..32) are
        // 256-position bitonic inputs whose runs of L are already sorted: odd
        // runs are laid out reversed and the network starts at runs of 2L
        const uint32_t L0 = __shfl_sync(LH_FULL, blen, 0);
        const bool has_q = q < ahi;
        const bool uniform = __all_sync(LH_FULL, !has_q || blen == L0) && L0 >= 4 && L0 <= 32 &&
                             (L0 & (L0 - 1)) == 0 && total <= kEscPairs;
        K key[8];
        if (uniform) {
            const uint32_t lg = 31 - __clz(L0);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t t = (lane << 3) + e;
                key[e] = ~K(0);
                if (t < total) {
                    const uint32_t r = t >> lg;
                    uint32_t off = t & (L0 - 1);
                    if (r & 1u) off = L0 - 1 - off;
                    const uint32_t pos = S.jb[r] + off;
                    float ph, pl;
                    lh_two_prod(S.ja[r], __ldg(bv + pos), ph, pl);
                    S.val[esc_vslot(t)] = make_float2(ph, pl);
                    key[e] = ((K)__ldg(B.lv[1].vals + pos) << 8) | t;
                }
            }
            switch (lg) {
                case 2: esc_sort256<K, 3>(key, lane); break;
                case 3: esc_sort256<K, 4>(key, lane); break;
                case 4: esc_sort256<K, 5>(key, lane); break;
                default: esc_sort256<K, 6>(key, lane); break;
            }
        } else {
            // expand: products 8 * lane + e
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t t = (lane << 3) + e;
                key[e] = ~K(0);
                if (t < total) {
                    uint32_t lo = 0, hi = 31;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (S.jp[mid] > t) hi = mid;
                        else lo = mid + 1;
                    }
                    const uint32_t pos = S.jb[lo] + (t - (S.jp[lo] - S.jl[lo]));
                    float ph, pl;
                    lh_two_prod(S.ja[lo], __ldg(bv + pos), ph, pl);
                    S.val[esc_vslot(t)] = make_float2(ph, pl);
                    key[e] = ((K)__ldg(B.lv[1].vals + pos) << 8) | t;
                }
            }
            esc_sort256(key, lane);
        }
        __syncwarp();
        // runs of equal k, in registers: sorted position 8 * lane + e holds key[e]
        uint32_t col[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) col[e] = (uint32_t)(key[e] >> 8);
        const uint32_t prev_last = __shfl_up_sync(LH_FULL, col[7], 1);
        uint32_t hmask = 0;  // bit e: position 8 * lane + e opens a run
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t ps = (lane << 3) + e;
            const uint32_t prev = e ? col[e - 1] : prev_last;
            if (ps < total && (ps == 0 || col[e] != prev)) hmask |= 1u << e;
        }
        const uint32_t heads = __popc(hmask);
        uint32_t hincl = heads;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(LH_FULL, hincl, o);
            if (lane >= o) hincl += t;
        }
        uint32_t oi = hincl - heads;
        // within the lane: runs it opens and closes are written at once; the
        // part before its first head is its lead, the open run its trail
        float ah = 0.f, al = 0.f, lead_h = 0.f, lead_l = 0.f;
        uint32_t rc = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float2 v = make_float2(0.f, 0.f);
            if ((lane << 3) + e < total) v = S.val[esc_vslot((uint32_t)(key[e] & 255u))];
            if ((hmask >> e) & 1u) {
                if (hmask & ((1u << e) - 1u)) {
                    ocol[oi] = rc;
                    oval[oi] = ah + al;
                    ++oi;
                } else {
                    lead_h = ah;
                    lead_l = al;
                }
                rc = col[e];
                ah = v.x;
                al = v.y;
            } else {
                lh_pair_add(ah, al, v.x, v.y);
            }
        }
        if (!hmask) {
            lead_h = ah;
            lead_l = al;
        }
        // segmented suffix sum of leads: q(L) = lead(L) + lead(L+1) + ... up to
        // and including the first lane at or after L that opens a run
        float qh = lead_h, ql = lead_l;
        int stop = hmask != 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float oh = __shfl_down_sync(LH_FULL, qh, o);
            const float ol = __shfl_down_sync(LH_FULL, ql, o);
            const int ostop = __shfl_down_sync(LH_FULL, stop, o);
            if (lane + o < 32 && !stop) {
                lh_pair_add(qh, ql, oh, ol);
                stop = ostop;
            }
        }
        // the lane's open run continues through the leads of the lanes after it
        float rh = __shfl_down_sync(LH_FULL, qh, 1), rl = __shfl_down_sync(LH_FULL, ql, 1);
        if (hmask) {
            if (lane < 31) lh_pair_add(ah, al, rh, rl);
            ocol[oi] = rc;
            oval[oi] = ah + al;
        }
        return __shfl_sync(LH_FULL, hincl, 31);
}

template <class K>
__global__ void __launch_bounds__(kEscWarps * 32, 6) k_spgemm_esc(
    DTrie A, const float *av, DTrie B, const float *bv, uint32_t nA0, const uint32_t *ub,
    const uint64_t *tmp_off, uint32_t *tcol, float *tval, uint32_t *cnt) {
    __shared__ EscSmem sm_all[kEscWarps];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    EscSmem &S = sm_all[warp];
    const uint32_t gw = blockIdx.x * kEscWarps + warp;
    const uint32_t nw = gridDim.x * kEscWarps;
    for (uint32_t p = gw; p < nA0; p += nw) {
        const uint32_t alo = __ldg(A.lv[0].offs + p), ahi = __ldg(A.lv[0].offs + p + 1);
        if (__ldg(ub + p) > kEscPairs || ahi - alo > 32) continue;
        const uint64_t t0 = tmp_off[p];
        const uint32_t n = esc_row<K>(A, av, B, bv, p, S, lane, tcol + t0, tval + t0);
        if (lane == 0) cnt[p] = n;
        __syncwarp();
    }
}

__global__ void k_spgemm_gather(uint32_t nA0, const uint64_t *tmp_off, const uint64_t *c_off,
                                const uint32_t *tcol, const float *tval, uint32_t *ccol, float *cval) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t p = gw; p < nA0; p += nw) {
        const uint64_t s0 = tmp_off[p], d0 = c_off[p], n = c_off[p + 1] - d0;
        // four strided positions per lane: all loads issued before the stores
        for (uint64_t s = lane; s < n; s += 128) {
            uint32_t c[4];
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t i = s + 32 * u;
                c[u] = i < n ? tcol[s0 + i] : 0u;
                v[u] = i < n ? tval[s0 + i] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t i = s + 32 * u;
                if (i < n) {
                    ccol[d0 + i] = c[u];
                    cval[d0 + i] = v[u];
                }
            }
        }
    }
}

}  // namespace

lh_status lh_run_spmv(lh_ctx *ctx, const lh_trie *a, const float *x, uint64_t x_n, uint64_t nrows,
                      lh_result *r) {
    if (a->nlevels != 2 || a->nannos < 1 || a->anno_type[0] != LH_T_F32)
        return lh_fail(ctx, LH_EINVAL, "SpMV needs a 2-level trie with an f32 annotation");
    if (x_n >= (1ull << 32) || nrows >= (1ull << 32)) return lh_fail(ctx, LH_EOVERFLOW, "SpMV sizes");
    r->nrows = nrows;
    LH_TRY(res_alloc(ctx, r, &r->y, nrows));
    LH_CU(cudaMemsetAsync(r->y, 0, nrows * sizeof(float), ctx->stream));
    const uint32_t n0 = (uint32_t)a->lv[0].n;
    if (n0 == 0) return LH_OK;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmv, kSpmvThreads, 0);
    unsigned grid = std::min<unsigned>(lh_blocks((uint64_t)n0 * kSpmvGroup, kSpmvThreads),
                                       (unsigned)(ctx->num_sms * std::max(1, per_sm)));
    LH_TRACED(ctx, "k_spmv", k_spmv<<<grid, kSpmvThreads, 0, ctx->stream>>>(lh_trie_dview(a), (const float *)a->anno[0], x,
                                                   (uint32_t)x_n, n0, r->y));
    LH_LAUNCH_CHECK();
    return LH_OK;
}

lh_status lh_run_spgemm(lh_ctx *ctx, const lh_trie *a, const lh_trie *b, lh_result *r, uint32_t dense_mode) {
    if (a->nlevels != 2 || b->nlevels != 2 || a->nannos < 1 || b->nannos < 1 ||
        a->anno_type[0] != LH_T_F32 || b->anno_type[0] != LH_T_F32)
        return lh_fail(ctx, LH_EINVAL, "SpGEMM needs 2-level tries with f32 annotations");
    const uint32_t n0 = (uint32_t)a->lv[0].n;
    const DTrie A = lh_trie_dview(a), B = lh_trie_dview(b);
    r->nrows = n0;
    r->c_row = a->lv[0].vals;
    LH_TRY(res_alloc(ctx, r, &r->c_off, (size_t)n0 + 1));
    uint32_t *ub = nullptr, *cnt = nullptr, *gkey = nullptr, *tcol = nullptr, *kmin = nullptr;
    uint8_t *kind = nullptr;
    uint64_t *tmp_off = nullptr, *gcap = nullptr, *goff = nullptr;
    unsigned long long *n_hash = nullptr;
    unsigned long long hash_rows = 0, dense_rows = 0;
    float *ghi = nullptr, *glo = nullptr, *tval = nullptr;
    lh_status s = LH_OK;
    uint64_t U = 0, G = 0;
    const unsigned T = 256;
    const unsigned grid = (unsigned)std::min<uint64_t>(lh_blocks(n0, T), (uint64_t)ctx->num_sms * 8);
#define STEP(x) if (s == LH_OK) s = (x)
    STEP(lh_alloc(ctx, &ub, n0));
    STEP(lh_alloc(ctx, &cnt, n0));
    STEP(lh_alloc(ctx, &tmp_off, (size_t)n0 + 1));
    STEP(lh_alloc(ctx, &gcap, n0));
    STEP(lh_alloc(ctx, &goff, (size_t)n0 + 1));
    STEP(lh_alloc(ctx, &n_hash, 3));
    STEP(lh_alloc(ctx, &kind, n0));
    STEP(lh_alloc(ctx, &kmin, n0));
    if (s == LH_OK && n0) {
        LH_TRACED(ctx, "k_spgemm_bound", k_spgemm_bound<<<grid, T, 0, ctx->stream>>>(A, B, n0, ub));
        cudaMemsetAsync(n_hash, 0, 3 * sizeof(unsigned long long), ctx->stream);
        LH_TRACED(ctx, "k_spgemm_gcap", k_spgemm_gcap<<<grid, T, 0, ctx->stream>>>(A, B, ub, n0, dense_mode, gcap, kind,
                                                                                 kmin, n_hash));
    }
    STEP(lh_scan_u32_to_u64(ctx, ub, tmp_off, n0));
    if (s == LH_OK && n0) {
        // U and the hash-row count in one readback
        LH_TRACED(ctx, "k_spgemm_sizes", k_spgemm_sizes<<<1, 32, 0, ctx->stream>>>(tmp_off + n0, n_hash));
        uint64_t h[3] = {0, 0, 0};
        STEP(lh_readback(ctx, n_hash, sizeof(h), h));
        U = h[0];
        hash_rows = h[1];
        dense_rows = h[2];
    }
    if (s == LH_OK && hash_rows) {
        // global hash tables only for rows whose products overflow shared memory
        STEP(lh_scan_u64_to_u64(ctx, gcap, goff, n0));
        STEP(lh_readback(ctx, goff + n0, sizeof(uint64_t), &G));
    }
    STEP(lh_alloc(ctx, &tcol, U));
    STEP(lh_alloc(ctx, &tval, U));
    STEP(lh_alloc(ctx, &gkey, G));
    STEP(lh_alloc(ctx, &ghi, G));
    STEP(lh_alloc(ctx, &glo, G));
    if (s == LH_OK && n0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spgemm_numeric, kGemmThreads, 0);
        unsigned g2 = (unsigned)std::min<uint64_t>((n0 + kGemmWarps - 1) / kGemmWarps,
                                                   (uint64_t)ctx->num_sms * std::max(1, per_sm));
        int per_sm_e = 0;
        const bool narrow = b->key_bits[1] <= 24;  // every k < 2^24
        if (narrow) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_e, k_spgemm_esc<uint32_t>, kEscWarps * 32, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_e, k_spgemm_esc<uint64_t>, kEscWarps * 32, 0);
        unsigned g3 = (unsigned)std::min<uint64_t>((n0 + kEscWarps - 1) / kEscWarps,
                                                   (uint64_t)ctx->num_sms * std::max(1, per_sm_e));
        if (dense_mode == 2) {
            // no sort kernel: its rows are dense or hashed
        } else if (narrow)
            LH_TRACED(ctx, "k_spgemm_esc", k_spgemm_esc<uint32_t><<<g3, kEscWarps * 32, 0, ctx->stream>>>(
                A, (const float *)a->anno[0], B, (const float *)b->anno[0], n0, ub, tmp_off, tcol, tval, cnt));
        else
            LH_TRACED(ctx, "k_spgemm_esc", k_spgemm_esc<uint64_t><<<g3, kEscWarps * 32, 0, ctx->stream>>>(
                A, (const float *)a->anno[0], B, (const float *)b->anno[0], n0, ub, tmp_off, tcol, tval, cnt));
        if (hash_rows) LH_TRACED(ctx, "k_spgemm_numeric", k_spgemm_numeric<<<g2, kGemmThreads, 0, ctx->stream>>>(A, (const float *)a->anno[0], B,
                                                               (const float *)b->anno[0], n0, tmp_off,
                                                               goff, gkey, ghi, glo, tcol, tval, cnt, kind,
                                                               dense_mode == 2 ? 1u : 0u));
        if (dense_rows) {
            const size_t smem = sizeof(DenseSmem);
            cudaFuncSetAttribute(k_spgemm_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per_sm_d = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_d, k_spgemm_dense, kDenseThreads, smem);
            const unsigned g4 = (unsigned)std::min<uint64_t>(n0, (uint64_t)ctx->num_sms * std::max(1, per_sm_d));
            LH_TRACED(ctx, "k_spgemm_dense", k_spgemm_dense<<<g4, kDenseThreads, smem, ctx->stream>>>(
                A, (const float *)a->anno[0], B, (const float *)b->anno[0], n0, kind, kmin, tmp_off, tcol, tval, cnt));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "spgemm: %s", cudaGetErrorString(e));
    }
    STEP(lh_scan_u32_to_u64(ctx, cnt, r->c_off, n0));
    // C is allocated at the product bound U, so no readback is needed here:
    // nnz = c_off[nrows] is read when the result is waited on
    STEP(res_alloc(ctx, r, &r->c_col, std::max<uint64_t>(U, 1)));
    STEP(res_alloc(ctx, r, &r->c_val, std::max<uint64_t>(U, 1)));
    if (s == LH_OK) r->nnz_pending = true;
    if (s == LH_OK && n0)
        LH_TRACED(ctx, "k_spgemm_gather", k_spgemm_gather<<<grid, T, 0, ctx->stream>>>(n0, tmp_off, r->c_off, tcol, tval, r->c_col, r->c_val));
#undef STEP
    lh_free(ctx, ub); lh_free(ctx, cnt); lh_free(ctx, tmp_off); lh_free(ctx, gcap); lh_free(ctx, goff);
    lh_free(ctx, n_hash); lh_free(ctx, kind); lh_free(ctx, kmin);
    lh_free(ctx, tcol); lh_free(ctx, tval); lh_free(ctx, gkey); lh_free(ctx, ghi); lh_free(ctx, glo);
    if (s == LH_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "spgemm: %s", cudaGetErrorString(e));
    }
    return s;
}
