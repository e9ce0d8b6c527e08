// Internal definitions shared by the CUDA translation units of liblh.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lh.h"

#define LH_WARP 32
#define LH_FULL 0xFFFFFFFFu
#define LH_NOSLOT 0xFFFFFFFFu

// ------------------------------------------------------------------ context

struct lh_trace_rec {
    const char *name;
    cudaEvent_t ev0, ev1;
};

struct lh_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 148;
    std::string err;
    cudaMemPool_t pool = nullptr;   // private stream-ordered pool (keeps its memory)
    bool user_alloc = false;        // device memory through the caller's allocator
    lh_alloc_fns fns{};
    uint32_t *d_status = nullptr;   // first device-side error (lh_status), 0 = none
    uint64_t *h_pinned = nullptr;   // pinned host words for small read-backs
    static constexpr int kPinnedWords = 64;
    // kernel tracing: CUDA events recorded on the launching stream around launches
    bool trace_on = false;
    std::string trace_only;         // when set, events bracket only this kernel
    std::vector<cudaEvent_t> ev_pool;
    std::vector<lh_trace_rec> pending;
    std::map<std::string, std::pair<uint64_t, double>> totals;
};

// Scoped trace of one kernel launch (no-op unless tracing is on).
struct LhTraceScope {
    lh_ctx *ctx;
    lh_trace_rec rec;
    bool on;
    LhTraceScope(lh_ctx *c, const char *name);
    ~LhTraceScope();
};

#define LH_TRACED(ctx_, name_, ...)              \
    do {                                         \
        LhTraceScope lh_scope_((ctx_), (name_)); \
        __VA_ARGS__;                             \
    } while (0)

lh_status lh_fail(lh_ctx *ctx, lh_status s, const char *fmt, ...);

#define LH_CU(call)                                                                     \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return lh_fail(ctx, e_ == cudaErrorMemoryAllocation ? LH_ENOMEM : LH_ECUDA, \
                           "%s: %s", #call, cudaGetErrorString(e_));                    \
    } while (0)

#define LH_TRY(expr)                 \
    do {                             \
        lh_status s_ = (expr);       \
        if (s_ != LH_OK) return s_;  \
    } while (0)

#define LH_LAUNCH_CHECK() LH_CU(cudaGetLastError())

// Stream-ordered device allocation on the context stream.
template <class T>
static inline lh_status lh_alloc(lh_ctx *ctx, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (ctx->user_alloc) {
        *p = (T *)ctx->fns.alloc((uint64_t)(count * sizeof(T)), (void *)ctx->stream, ctx->fns.user);
        if (!*p) return lh_fail(ctx, LH_ENOMEM, "caller's allocator refused %zu bytes", count * sizeof(T));
        return LH_OK;
    }
    cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync((void **)p, count * sizeof(T), ctx->pool, ctx->stream)
                              : cudaMallocAsync((void **)p, count * sizeof(T), ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return lh_fail(ctx, LH_ENOMEM, "cudaMallocAsync(%zu bytes): %s", count * sizeof(T),
                       cudaGetErrorString(e));
    }
    return LH_OK;
}
static inline void lh_free(lh_ctx *ctx, void *p) {
    if (!p) return;
    if (ctx->user_alloc) ctx->fns.free(p, (void *)ctx->stream, ctx->fns.user);
    else cudaFreeAsync(p, ctx->stream);
}

// Copy `n` 64-bit device words to the pinned buffer and wait for them.
lh_status lh_readback(lh_ctx *ctx, const void *dev, size_t bytes, void *host);

static inline unsigned lh_blocks(uint64_t n, unsigned threads, unsigned cap = 1u << 30) {
    uint64_t b = (n + threads - 1) / threads;
    if (b == 0) b = 1;
    return (unsigned)(b > cap ? cap : b);
}

// -------------------------------------------------------------------- scans

// out[i] = sum_{j<i} in[j] (exclusive), out[n] = total (out has n+1 slots).
lh_status lh_scan_u32_to_u64(lh_ctx *ctx, const uint32_t *in, uint64_t *out, uint64_t n);
lh_status lh_scan_u32_to_u32(lh_ctx *ctx, const uint32_t *in, uint32_t *out, uint64_t n);
lh_status lh_scan_u64_to_u64(lh_ctx *ctx, const uint64_t *in, uint64_t *out, uint64_t n);

// ----------------------------------------------------------------- radix sort

// Stable LSD radix sort of (key, val) pairs on the low `bits` bits of key.
// (*keys, *vals) hold the input and (*tmp_k, *tmp_v) scratch of length n; on
// return the pointers are swapped as needed so that (*keys, *vals) hold the
// sorted pairs and (*tmp_k, *tmp_v) the scratch.  status: a zeroed device
// word that receives LH_ETIMEOUT if a bounded wait gives up (the caller
// reads it back), or null for the sort to read its own back.  hist: the
// 256-bin digit counts of every pass (pass p at hist[256 p]) when the caller
// has counted them already, or null for the sort to count them.
lh_status lh_radix_sort_u64(lh_ctx *ctx, uint64_t **keys, uint32_t **vals, uint64_t **tmp_k,
                            uint32_t **tmp_v, uint64_t n, int bits, uint32_t *status,
                            const unsigned long long *hist = nullptr);

// ----------------------------------------------------------------------- tries

struct TrieLevel {
    uint64_t n = 0;       // entries
    uint64_t nsets = 0;   // sets (1 at level 0; entries of the previous level otherwise)
    uint32_t *vals = nullptr;
    uint32_t *offs = nullptr;     // n + 1 offsets into the next level (null at the leaf)
    uint32_t *bs_slot = nullptr;  // nsets, or null when the level has no bitset set
    uint64_t n_bs = 0;
    uint32_t *bs_meta = nullptr;  // 4 * n_bs: first word, base, words, card
};

struct lh_trie {
    uint32_t nlevels = 0;
    uint32_t key_order[LH_MAX_LEVELS] = {0};
    uint32_t key_bits[LH_MAX_LEVELS] = {0};  // bits of the largest value per level
    uint64_t nrows_in = 0;
    TrieLevel lv[LH_MAX_LEVELS];
    uint32_t *words = nullptr;
    uint32_t *rank = nullptr;
    uint64_t nwords = 0;
    uint32_t nannos = 0;
    void *anno[LH_MAX_ANNOS] = {nullptr};
    uint32_t anno_type[LH_MAX_ANNOS] = {0};
    uint32_t bs_ratio = 0, bs_min_card = 0;
    uint32_t level_ratio[LH_MAX_LEVELS] = {0};   // layout ratio of each level (0 = uint only)
    uint64_t bytes = 0;
    std::vector<void *> allocs;
};

// Device view of a trie (passed by value to kernels).
struct DLevel {
    const uint32_t *vals;
    const uint32_t *offs;
    const uint32_t *bs_slot;
    const uint4 *bs_meta;
    uint32_t n;
};

struct DTrie {
    DLevel lv[LH_MAX_LEVELS];
    const uint32_t *words;
    const uint32_t *rank;
    uint32_t nlevels;
};

DTrie lh_trie_dview(const lh_trie *t);

// Decide layouts and emit bitsets for every level of a trie whose vals/offs
// are complete (shared by the relation and filter builders).
lh_status lh_trie_layout(lh_ctx *ctx, lh_trie *t);
void lh_trie_release(lh_ctx *ctx, lh_trie *t);

// ------------------------------------------------------- device set helpers

// Range [lo, hi) of the set at level L whose parent entry is `parent`
// (ignored at level 0).
__device__ __forceinline__ void lh_set_range(const DTrie &T, int L, uint32_t parent, uint32_t &lo,
                                             uint32_t &hi) {
    if (L == 0) {
        lo = 0;
        hi = T.lv[0].n;
    } else {
        const uint32_t *o = T.lv[L - 1].offs;
        lo = __ldg(o + parent);
        hi = __ldg(o + parent + 1);
    }
}

// First index in vals[lo, hi) with vals[idx] >= x.
__device__ __forceinline__ uint32_t lh_lower_bound(const uint32_t *vals, uint32_t lo, uint32_t hi,
                                                   uint32_t x) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(vals + mid) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Membership of x in the set (level L, set index `set`, range [lo, hi)).  On
// success *pos is x's index in the level's vals.  Bitset sets answer with one
// word load and a rank; uint sets with a binary search.
__device__ __forceinline__ bool lh_probe(const DTrie &T, int L, uint32_t set, uint32_t lo,
                                         uint32_t hi, uint32_t x, uint32_t *pos) {
    const DLevel &lv = T.lv[L];
    if (lv.bs_slot != nullptr) {
        uint32_t slot = __ldg(lv.bs_slot + set);
        if (slot != LH_NOSLOT) {
            uint4 m = __ldg(lv.bs_meta + slot);  // first word, base, words, rank base
            if (x < m.y) return false;
            uint32_t d = x - m.y;
            uint32_t w = d >> 5;
            if (w >= m.z) return false;
            uint32_t word = __ldg(T.words + m.x + w);
            uint32_t b = d & 31u;
            if (!((word >> b) & 1u)) return false;
            *pos = lo + (__ldg(T.rank + m.x + w) - m.w) + __popc(word & ((1u << b) - 1u));
            return true;
        }
    }
    uint32_t p = lh_lower_bound(lv.vals, lo, hi, x);
    if (p < hi && __ldg(lv.vals + p) == x) {
        *pos = p;
        return true;
    }
    return false;
}

// Compensated fp32 arithmetic (error-free transformations).
__device__ __forceinline__ void lh_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void lh_two_prod(float a, float b, float &p, float &e) {
    p = a * b;
    e = fmaf(a, b, -p);
}
// (sh, sl) += (th, tl)
__device__ __forceinline__ void lh_pair_add(float &sh, float &sl, float th, float tl) {
    float s, e;
    lh_two_sum(sh, th, s, e);
    sh = s;
    sl += e + tl;
}

__device__ __forceinline__ void lh_set_status(uint32_t *st, uint32_t code) {
    atomicCAS(st, 0u, code);
}
