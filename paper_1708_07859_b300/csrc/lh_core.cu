// Context, error reporting, device scans and the LSD radix sort used by the
// trie builder (Section 2.2: tries are built from sorted key tuples).
#include "lh_internal.cuh"

lh_status lh_fail(lh_ctx *ctx, lh_status s, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

static void trace_fold(lh_ctx *ctx);

extern "C" const char *lh_version(void) { return "lh-b300 0.1 (sm_103a)"; }

static lh_status create_ctx(lh_ctx **out, void *stream, const lh_alloc_fns *fns) {
    if (!out) return LH_EINVAL;
    *out = nullptr;
    lh_ctx *ctx = new lh_ctx();
    ctx->stream = (cudaStream_t)stream;
    if (fns) {
        ctx->user_alloc = true;
        ctx->fns = *fns;
    }
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess && !fns) {
        // a private pool whose memory stays mapped between calls: the default
        // pool would hand multi-GB temporaries back at every synchronisation
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        e = cudaMemPoolCreate(&ctx->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e == cudaSuccess) {
        if (fns) {
            ctx->d_status = (uint32_t *)fns->alloc(sizeof(uint32_t), stream, fns->user);
            if (!ctx->d_status) e = cudaErrorMemoryAllocation;
        } else {
            e = cudaMalloc((void **)&ctx->d_status, sizeof(uint32_t));
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&ctx->h_pinned, lh_ctx::kPinnedWords * sizeof(uint64_t),
                          cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_status) {
            if (fns) fns->free(ctx->d_status, stream, fns->user);
            else cudaFree(ctx->d_status);
        }
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        delete ctx;
        return LH_ECUDA;
    }
    *out = ctx;
    return LH_OK;
}

extern "C" lh_status lh_create(lh_ctx **out, void *stream) { return create_ctx(out, stream, nullptr); }

extern "C" lh_status lh_create_with_allocator(lh_ctx **out, void *stream, const lh_alloc_fns *fns) {
    if (!fns || !fns->alloc || !fns->free) return LH_EINVAL;
    return create_ctx(out, stream, fns);
}

extern "C" lh_status lh_destroy(lh_ctx *ctx) {
    if (!ctx) return LH_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    trace_fold(ctx);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->d_status) {
        if (ctx->user_alloc) ctx->fns.free(ctx->d_status, (void *)ctx->stream, ctx->fns.user);
        else cudaFree(ctx->d_status);
    }
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->pool) {
        cudaDeviceSynchronize();  // memory freed asynchronously must be released before the pool goes
        cudaMemPoolDestroy(ctx->pool);
    }
    delete ctx;
    return LH_OK;
}

extern "C" lh_status lh_pool_reserve(lh_ctx *ctx, uint64_t bytes) {
    if (!ctx) return LH_EINVAL;
    if (ctx->user_alloc) return lh_fail(ctx, LH_EUNSUPPORTED, "the context uses the caller's allocator");
    if (!ctx->pool) return LH_EINVAL;
    if (bytes == 0) return LH_OK;
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, ctx->pool, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return lh_fail(ctx, LH_ENOMEM, "pool reserve of %llu bytes: %s", (unsigned long long)bytes,
                       cudaGetErrorString(e));
    }
    LH_CU(cudaFreeAsync(p, ctx->stream));
    LH_CU(cudaStreamSynchronize(ctx->stream));
    return LH_OK;
}

extern "C" lh_status lh_pool_usage(lh_ctx *ctx, uint64_t *used_now, uint64_t *used_high, int reset_high) {
    if (!ctx) return LH_EINVAL;
    if (ctx->user_alloc) return lh_fail(ctx, LH_EUNSUPPORTED, "the context uses the caller's allocator");
    if (!ctx->pool) return LH_EINVAL;
    unsigned long long now = 0, high = 0;  // the pool attributes are 64-bit
    LH_CU(cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, &now));
    LH_CU(cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &high));
    if (used_now) *used_now = now;
    if (used_high) *used_high = high;
    if (reset_high) {
        unsigned long long zero = 0;  // resets the high-water mark to the current use
        LH_CU(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    return LH_OK;
}

extern "C" lh_status lh_set_stream(lh_ctx *ctx, void *stream) {
    if (!ctx) return LH_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return LH_OK;
}

extern "C" const char *lh_last_error(const lh_ctx *ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" lh_status lh_sync(lh_ctx *ctx) {
    if (!ctx) return LH_EINVAL;
    LH_CU(cudaStreamSynchronize(ctx->stream));
    uint32_t st = 0;
    LH_CU(cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st != 0) {
        LH_CU(cudaMemset(ctx->d_status, 0, sizeof(uint32_t)));
        const char *what = st == LH_EINVAL      ? "a value outside its declared domain (key bound or GROUP BY card)"
                           : st == LH_ETIMEOUT   ? "a bounded wait gave up"
                           : st == LH_EOVERFLOW  ? "a 32-bit offset or capacity overflowed"
                                                 : "error";
        return lh_fail(ctx, (lh_status)st, "device-side error %u: %s", st, what);
    }
    return LH_OK;
}

extern "C" lh_status lh_copy_d2h(lh_ctx *ctx, void *host, const void *dev, uint64_t bytes) {
    if (!ctx || (bytes && (!host || !dev))) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (!bytes) return LH_OK;
    LH_CU(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    LH_CU(cudaStreamSynchronize(ctx->stream));
    return LH_OK;
}

extern "C" lh_status lh_copy_h2d(lh_ctx *ctx, void *dev, const void *host, uint64_t bytes) {
    if (!ctx || (bytes && (!host || !dev))) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (!bytes) return LH_OK;
    LH_CU(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    LH_CU(cudaStreamSynchronize(ctx->stream));
    return LH_OK;
}

// ------------------------------------------------------------------ tracing

static cudaEvent_t pool_event(lh_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

LhTraceScope::LhTraceScope(lh_ctx *c, const char *name) : ctx(c), on(c && c->trace_on) {
    if (!on) return;
    if (!ctx->trace_only.empty() && ctx->trace_only != name) {
        ctx->totals[name].first += 1;  // counted, not timed
        on = false;
        return;
    }
    rec.name = name;
    rec.ev0 = pool_event(ctx);
    rec.ev1 = pool_event(ctx);
    cudaEventRecord(rec.ev0, ctx->stream);
}

LhTraceScope::~LhTraceScope() {
    if (!on) return;
    cudaEventRecord(rec.ev1, ctx->stream);
    ctx->pending.push_back(rec);
}

static void trace_fold(lh_ctx *ctx) {
    for (auto &r : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.ev0, r.ev1) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        auto &t = ctx->totals[r.name];
        t.first += 1;
        t.second += ms;
        ctx->ev_pool.push_back(r.ev0);
        ctx->ev_pool.push_back(r.ev1);
    }
    ctx->pending.clear();
}

extern "C" lh_status lh_trace_enable(lh_ctx *ctx, int on) {
    if (!ctx) return LH_EINVAL;
    ctx->trace_on = on != 0;
    return LH_OK;
}

extern "C" lh_status lh_trace_only(lh_ctx *ctx, const char *name) {
    if (!ctx) return LH_EINVAL;
    ctx->trace_only = name ? name : "";
    return LH_OK;
}

extern "C" lh_status lh_trace_read(lh_ctx *ctx, lh_trace_entry *out, uint32_t cap, uint32_t *n) {
    if (!ctx || !n || (cap && !out)) return lh_fail(ctx, LH_EINVAL, "null argument");
    LH_CU(cudaStreamSynchronize(ctx->stream));
    trace_fold(ctx);
    uint32_t k = 0;
    for (auto &kv : ctx->totals) {
        if (k < cap) {
            memset(&out[k], 0, sizeof(out[k]));
            strncpy(out[k].name, kv.first.c_str(), sizeof(out[k].name) - 1);
            out[k].launches = kv.second.first;
            out[k].total_ms = kv.second.second;
        }
        ++k;
    }
    *n = k;
    return LH_OK;
}

extern "C" lh_status lh_trace_reset(lh_ctx *ctx) {
    if (!ctx) return LH_EINVAL;
    LH_CU(cudaStreamSynchronize(ctx->stream));
    trace_fold(ctx);
    ctx->totals.clear();
    return LH_OK;
}

lh_status lh_readback(lh_ctx *ctx, const void *dev, size_t bytes, void *host) {
    if (bytes > lh_ctx::kPinnedWords * sizeof(uint64_t))
        return lh_fail(ctx, LH_EINVAL, "readback too large");
    LH_CU(cudaMemcpyAsync(ctx->h_pinned, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    LH_CU(cudaStreamSynchronize(ctx->stream));
    memcpy(host, ctx->h_pinned, bytes);
    return LH_OK;
}

// ---------------------------------------------------------------------- scan
// Three-phase exclusive scan: per-tile sums, a scan of the tile sums
// (recursive), then a rescan of every tile seeded with its prefix.

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class TO>
__device__ TO block_exclusive_scan(TO v, TO *warp_tot, TO &block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TO incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        TO t = __shfl_up_sync(LH_FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        TO w = lane < (kScanThreads / 32) ? warp_tot[lane] : TO(0);
        TO wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            TO t = __shfl_up_sync(LH_FULL, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = wi - w;
        if (lane == (kScanThreads / 32) - 1) warp_tot[kScanThreads / 32] = wi;
    }
    __syncthreads();
    TO r = warp_tot[warp] + incl - v;
    block_total = warp_tot[kScanThreads / 32];
    __syncthreads();
    return r;
}

template <class TI, class TO>
__global__ void k_tile_sums(const TI *in, uint64_t n, TO *sums) {
    __shared__ TO wt[kScanThreads / 32 + 1];
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    TO s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += (TO)in[base + k];
    TO tot;
    block_exclusive_scan<TO>(s, wt, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <class TI, class TO>
__global__ void k_tile_scan(const TI *in, uint64_t n, const TO *prefix, TO *out) {
    __shared__ TO wt[kScanThreads / 32 + 1];
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    TO v[kScanItems];
    TO s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? (TO)in[base + k] : TO(0);
        s += v[k];
    }
    TO tot;
    TO run = block_exclusive_scan<TO>(s, wt, tot) + (prefix ? prefix[blockIdx.x] : TO(0));
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    // the thread holding the last element also writes the grand total
    if (base < n && base + kScanItems >= n) out[n] = run;
}

template <class TI, class TO>
lh_status scan_impl(lh_ctx *ctx, const TI *in, TO *out, uint64_t n) {
    if (n == 0) {
        LH_CU(cudaMemsetAsync(out, 0, sizeof(TO), ctx->stream));
        return LH_OK;
    }
    uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        LH_TRACED(ctx, "k_tile_scan", k_tile_scan<TI, TO><<<1, kScanThreads, 0, ctx->stream>>>(in, n, (const TO *)nullptr, out));
        LH_LAUNCH_CHECK();
        return LH_OK;
    }
    TO *sums = nullptr, *pref = nullptr;
    LH_TRY(lh_alloc(ctx, &sums, tiles));
    if (lh_status s0 = lh_alloc(ctx, &pref, tiles + 1); s0 != LH_OK) {
        lh_free(ctx, sums);
        return s0;
    }
    LH_TRACED(ctx, "k_tile_sums", k_tile_sums<TI, TO><<<(unsigned)tiles, kScanThreads, 0, ctx->stream>>>(in, n, sums));
    LH_LAUNCH_CHECK();
    lh_status s = scan_impl<TO, TO>(ctx, sums, pref, tiles);
    if (s == LH_OK) {
        LH_TRACED(ctx, "k_tile_scan", k_tile_scan<TI, TO><<<(unsigned)tiles, kScanThreads, 0, ctx->stream>>>(in, n, pref, out));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "scan: %s", cudaGetErrorString(e));
    }
    lh_free(ctx, sums);
    lh_free(ctx, pref);
    return s;
}

}  // namespace

lh_status lh_scan_u32_to_u64(lh_ctx *ctx, const uint32_t *in, uint64_t *out, uint64_t n) {
    return scan_impl<uint32_t, uint64_t>(ctx, in, out, n);
}
lh_status lh_scan_u32_to_u32(lh_ctx *ctx, const uint32_t *in, uint32_t *out, uint64_t n) {
    return scan_impl<uint32_t, uint32_t>(ctx, in, out, n);
}
lh_status lh_scan_u64_to_u64(lh_ctx *ctx, const uint64_t *in, uint64_t *out, uint64_t n) {
    return scan_impl<uint64_t, uint64_t>(ctx, in, out, n);
}

// ---------------------------------------------------------------- radix sort
// LSD, 8-bit digits, one kernel per pass.  One upfront kernel reads the keys
// once and counts the digits of every pass (global 256-bin histograms); a
// pass's digit d then starts at the exclusive prefix of its histogram.
// Within a pass, tiles of 3072 keys are taken in ticket order; each tile
// ranks its keys in shared memory, publishes its per-digit counts, and
// finds, for every digit, the count of that digit in all earlier tiles by
// decoupled look-back (thread d walks back over earlier tiles' states until
// one carries an inclusive prefix).  Every tile waited on was ticketed
// earlier, so it is already running and publishes its counts without
// waiting.  The scatter is stable: ranks follow key order within a tile,
// and tiles follow key order.

namespace {

constexpr int kSortThreads = 256;
// 12 rounds of 256 keys: 3072-key tiles at 64 registers a thread fit four
// CTAs per SM (16 rounds at three CTAs measured 1.57 ms per step against 1.51)
constexpr int kSortRounds = 12;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 3072 keys per tile
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortMaxPasses = 8;
constexpr unsigned long long kSortAgg = 1ull << 62, kSortInc = 1ull << 63, kSortVal = (1ull << 62) - 1;
constexpr uint32_t kSortSpins = 1u << 20;

// digit histograms of every pass, one read of the keys
__global__ void k_sort_upsweep(const uint64_t *keys, uint64_t n, int passes, unsigned long long *ghist) {
    __shared__ uint32_t h[kSortMaxPasses][256];
    for (int i = threadIdx.x; i < kSortMaxPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 4 * stride) {
        uint64_t k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) k[u] = i + u * stride < n ? keys[i + u * stride] : 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i + u * stride >= n) break;
            for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k[u] >> (8 * p)) & 255u], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(ghist + i, (unsigned long long)c);
    }
}

__device__ __forceinline__ void sort_store(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long sort_load(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// lanes holding the same 9-bit label (digit 0..255, or 256 for no key):
// one ballot per label bit, keeping the lanes that agree on it
__device__ __forceinline__ uint32_t match_label9(uint32_t d) {
    uint32_t peers = LH_FULL;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t m = __ballot_sync(LH_FULL, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// One pass over one tile.  Warp w ranks the tile's keys [w*384, (w+1)*384)
// in 12 rounds of 32 with warp-private digit counters (lanes with equal
// digits are grouped by one ballot per digit bit; the group's leader reads
// and advances the counter).  A prefix over warps and digits turns the
// counters into each (warp, digit) start in shared memory, where keys are
// placed grouped by digit and written out as contiguous per-digit runs.
constexpr size_t kScatterSmem = (size_t)kSortTile * (sizeof(uint64_t) + sizeof(uint32_t));

__global__ void __launch_bounds__(kSortThreads, 4) k_sort_onesweep(
    const uint64_t *kin, const uint32_t *vin, uint64_t n, int shift, const unsigned long long *ghist,
    unsigned long long *state, uint32_t *ticket, uint32_t *status, uint64_t *kout, uint32_t *vout) {
    extern __shared__ uint64_t s_keys[];                       // kSortTile keys, grouped by digit
    uint32_t *s_vals = (uint32_t *)(s_keys + kSortTile);      // their payloads
    __shared__ uint32_t wcnt[kSortWarps][256];                // per-warp digit counts, then starts
    __shared__ uint32_t lstart[256];
    __shared__ uint32_t wtot[kSortWarps];
    __shared__ uint64_t wtot64[kSortWarps];
    __shared__ uint64_t gbase[256];
    __shared__ uint32_t s_tile, s_ok;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) {
        s_tile = atomicAdd(ticket, 1u);
        // an earlier wait gave up: the keys no longer match the histograms
        s_ok = *(volatile uint32_t *)status == 0;
    }
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wcnt[w][t] = 0;
    __syncthreads();
    if (!s_ok) return;
    const uint32_t tile = s_tile;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint64_t tbase = (uint64_t)tile * kSortTile;
    const uint32_t tile_n = (uint32_t)min((uint64_t)kSortTile, n - tbase);
    const uint64_t wbase = tbase + (uint64_t)warp * (kSortRounds * 32);
    // all of this thread's keys are loaded up front: one memory latency per tile
    uint64_t kr[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const uint64_t i = wbase + (uint64_t)r * 32 + lane;
        kr[r] = i < n ? kin[i] : 0;
    }
    // where digit t starts in this pass's output: exclusive prefix of the histogram
    uint64_t dstart;
    {
        const uint64_t c = ghist[t];
        uint64_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t x = __shfl_up_sync(LH_FULL, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) wtot64[warp] = incl;
        __syncthreads();
        uint64_t wp = 0;
        for (int w = 0; w < warp; ++w) wp += wtot64[w];
        dstart = wp + incl - c;
    }
    uint32_t rk[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const bool valid = wbase + (uint64_t)r * 32 + lane < n;
        const uint32_t d = valid ? (uint32_t)((kr[r] >> shift) & 255u) : 256u;
        const uint32_t peers = match_label9(d);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && lane == leader) {
            before = wcnt[warp][d];
            wcnt[warp][d] = before + __popc(peers);
        }
        rk[r] = __shfl_sync(LH_FULL, before, leader) + __popc(peers & lt_mask);
        __syncwarp();
    }
    __syncthreads();
    // thread t owns digit t: exclusive prefix over warps and the tile's count,
    // published at once; then each digit's run start in shared memory
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t x = wcnt[w][t];
        wcnt[w][t] = c;
        c += x;
    }
    unsigned long long *st = state + (uint64_t)tile * 256 + t;
    sort_store(st, (tile == 0 ? kSortInc : kSortAgg) | c);
    {
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(LH_FULL, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        uint32_t wp = 0;
        for (int w = 0; w < warp; ++w) wp += wtot[w];
        const uint32_t start = wp + incl - c;
        lstart[t] = start;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wcnt[w][t] += start;
    }
    __syncthreads();
    // keys go to their slots first; the payloads are loaded only now, when
    // the keys' registers are free, and follow them
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        if (wbase + (uint64_t)r * 32 + lane < n) {
            const uint32_t d = (uint32_t)((kr[r] >> shift) & 255u);
            rk[r] += wcnt[warp][d];
            s_keys[rk[r]] = kr[r];
        }
    }
    uint32_t vr[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const uint64_t i = wbase + (uint64_t)r * 32 + lane;
        vr[r] = i < n ? vin[i] : 0;
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r)
        if (wbase + (uint64_t)r * 32 + lane < n) s_vals[rk[r]] = vr[r];
    {
        // the count of digit t in all earlier tiles, eight earlier tiles per
        // round trip: add the published counts up to the first inclusive
        // prefix; wait only where a count is missing
        uint64_t excl = 0;
        bool ok = true;
        uint32_t spins = 0;
        for (int64_t q = (int64_t)tile - 1; q >= 0;) {
            unsigned long long w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) w[j] = q - j >= 0 ? sort_load(state + (uint64_t)(q - j) * 256 + t) : kSortInc;
            int used = 0;
            bool done = false, missing = false;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (done || missing) continue;
                if ((w[j] >> 62) == 0) {
                    missing = true;
                    continue;
                }
                excl += w[j] & kSortVal;
                ++used;
                done = (w[j] & kSortInc) != 0;
            }
            if (done) break;
            q -= used;
            if (missing) {
                if (++spins >= kSortSpins || ((spins & 255u) == 0 && *(volatile uint32_t *)status)) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (tile > 0) sort_store(st, kSortInc | ((excl + c) & kSortVal));
        if (!ok) {
            lh_set_status(status, LH_ETIMEOUT);
            s_ok = 0;
        }
        gbase[t] = dstart + excl;
    }
    __syncthreads();
    if (!s_ok) return;
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const uint32_t at = r * kSortThreads + t;
        if (at < tile_n) {
            const uint64_t k = s_keys[at];
            const uint32_t d = (uint32_t)((k >> shift) & 255u);
            const uint64_t dst = gbase[d] + (at - lstart[d]);
            if (dst < n) {
                kout[dst] = k;
                vout[dst] = s_vals[at];
            }
        }
    }
}

}  // namespace

lh_status lh_radix_sort_u64(lh_ctx *ctx, uint64_t **keys, uint32_t **vals, uint64_t **tmp_k,
                            uint32_t **tmp_v, uint64_t n, int bits, uint32_t *status_out,
                            const unsigned long long *hist_in) {
    if (n <= 1 || bits <= 0) return LH_OK;
    const uint64_t ntiles64 = (n + kSortTile - 1) / kSortTile;
    if (ntiles64 > (1u << 24)) return lh_fail(ctx, LH_EUNSUPPORTED, "sort: too many keys");
    const uint32_t ntiles = (uint32_t)ntiles64;
    const int passes = (bits + 7) / 8;
    if (passes > kSortMaxPasses) return lh_fail(ctx, LH_EINVAL, "sort: more than 64 key bits");
    // one zeroed block: histograms (unless the caller counted them), look-back
    // states, tickets, status
    const size_t n_hist = hist_in ? 0 : (size_t)passes * 256, n_state = (size_t)passes * ntiles * 256;
    const size_t words = n_hist + n_state + (size_t)(passes + 2) / 2 + 1;
    unsigned long long *scratch = nullptr;
    LH_TRY(lh_alloc(ctx, &scratch, words));
    unsigned long long *ghist = scratch, *state = scratch + n_hist;
    uint32_t *tickets = (uint32_t *)(state + n_state);
    uint32_t *status = status_out ? status_out : tickets + passes;
    lh_status s = LH_OK;
    {
        cudaError_t e = cudaMemsetAsync(scratch, 0, words * sizeof(unsigned long long), ctx->stream);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sort_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "sort setup: %s", cudaGetErrorString(e));
    }
    if (s == LH_OK && !hist_in) {
        const unsigned g = (unsigned)std::min<uint64_t>(lh_blocks((n + 3) / 4, 256), (uint64_t)ctx->num_sms * 8);
        LH_TRACED(ctx, "k_sort_upsweep", k_sort_upsweep<<<g, 256, 0, ctx->stream>>>(*keys, n, passes, ghist));
    }
    const unsigned long long *hist = hist_in ? hist_in : ghist;
    uint64_t *ka = *keys, *kb = *tmp_k;
    uint32_t *va = *vals, *vb = *tmp_v;
    for (int p = 0; p < passes && s == LH_OK; ++p) {
        LH_TRACED(ctx, "k_sort_onesweep", k_sort_onesweep<<<ntiles, kSortThreads, kScatterSmem, ctx->stream>>>(
                                              ka, va, n, 8 * p, hist + (size_t)p * 256,
                                              state + (size_t)p * ntiles * 256, tickets + p, status, kb, vb));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "sort: %s", cudaGetErrorString(e));
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    // the sorted data stays where the last pass wrote it: hand back the buffers
    *keys = ka;
    *tmp_k = kb;
    *vals = va;
    *tmp_v = vb;
    if (s == LH_OK && !status_out) {
        uint32_t st = 0;
        s = lh_readback(ctx, status, sizeof(st), &st);
        if (s == LH_OK && st) s = lh_fail(ctx, (lh_status)st, "sort: look-back wait gave up");
    }
    lh_free(ctx, scratch);
    return s;
}
