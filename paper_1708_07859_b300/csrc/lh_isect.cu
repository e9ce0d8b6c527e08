// Count-only set intersection of many independent pairs (the core operation
// of an attribute, Section 2.4; the three layout pairs of Section 4.1.1 /
// Figure 4a).  All pairs are cut into fixed-size tiles; merge tiles are
// drained by one launch of k_isect4 (shared staging), the other kinds by one
// launch of k_isect_lean (no staging, higher occupancy):
//   uint cap uint, sizes within 32x: merge path.  Tile t covers diagonals
//     [t*TILE, (t+1)*TILE) of the pair's merge; the A and B slices it
//     consumes are staged in shared memory and every thread merges 16
//     diagonals.  A match is counted when its A element is consumed and the
//     current B head equals it, so each is counted exactly once.
//   uint cap uint, sizes beyond 32x: every element of the smaller set is
//     binary-searched in the larger.
//   uint cap bs: every uint element tests one bit.
//   bs cap bs: 128-bit word AND + popc over the overlapping word range.
#include <mutex>

#include "lh_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // merge diagonals (or elements, or words) per tile

enum { K_MERGE = 0, K_PROBE = 1, K_UBS = 2, K_BB = 3, K_EMPTY = 4 };

struct PairPlan {
    uint32_t kind;
    uint32_t swap;  // 1: roles of a and b exchanged
    uint64_t lo_w, hi_w;  // bs cap bs: absolute word range of the overlap
};

__device__ __forceinline__ uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

__global__ void k_plan(uint32_t npairs, const lh_set *A, const lh_set *B, PairPlan *plan,
                       uint64_t *tiles, unsigned long long *n_merge = nullptr) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    lh_set a = A[p], b = B[p];
    PairPlan pl = {K_EMPTY, 0, 0, 0};
    uint64_t nt = 0;
    if (a.n > 0 && b.n > 0) {
        if (a.layout == 0 && b.layout == 0) {
            uint64_t mn = min(a.n, b.n), mx = max(a.n, b.n);
            // the merge closes its slices with 0xFFFFFFFF sentinels
            const bool max_val = a.data[a.n - 1] == 0xFFFFFFFFu || b.data[b.n - 1] == 0xFFFFFFFFu;
            if (mx <= 32 * mn && !max_val) {
                pl.kind = K_MERGE;
                nt = ceil_div(a.n + b.n, kTile);
            } else {
                pl.kind = K_PROBE;
                pl.swap = a.n > b.n;
                nt = ceil_div(mn, kTile);
            }
        } else if (a.layout == 1 && b.layout == 1) {
            uint64_t a0 = a.base >> 5, b0 = b.base >> 5;
            uint64_t lo = max(a0, b0), hi = min(a0 + a.n, b0 + b.n);
            if (hi > lo) {
                pl.kind = K_BB;
                pl.lo_w = lo;
                pl.hi_w = hi;
                nt = ceil_div(hi - lo, kTile);
            }
        } else {
            pl.kind = K_UBS;
            pl.swap = a.layout == 1;  // the uint side goes first
            nt = ceil_div(a.layout == 0 ? a.n : b.n, kTile);
        }
    }
    plan[p] = pl;
    tiles[p] = nt;
    if (n_merge && pl.kind == K_MERGE && nt) atomicAdd(n_merge, (unsigned long long)nt);
}

// merge-path split of diagonal d (ties: A first)
__device__ __forceinline__ uint64_t mp_split(const uint32_t *a, uint64_t na, const uint32_t *b,
                                             uint64_t nb, uint64_t d) {
    uint64_t lo = d > nb ? d - nb : 0, hi = min(d, na);
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) <= __ldg(b + d - mid - 1)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t sm_split(const uint32_t *a, uint32_t na, const uint32_t *b,
                                             uint32_t nb, uint32_t d) {
    uint32_t lo = d > nb ? d - nb : 0, hi = min(d, na);
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= b[d - mid - 1]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LH_FULL, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(LH_FULL, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// pair of a global tile: last p with tile_off[p] <= tile
__device__ __forceinline__ uint32_t tile_pair(const uint64_t *tile_off, uint32_t npairs, uint64_t tile) {
    uint32_t lo = 0, hi = npairs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (tile_off[mid] <= tile) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Tile loop of the allocation-free entry point: every tile finds its pair and
// its merge-path splits itself (no per-tile descriptors, which would need an
// allocation sized by the tile count).
__global__ void __launch_bounds__(kThreads) k_isect(uint32_t npairs, const lh_set *A,
                                                    const lh_set *B, const PairPlan *plan,
                                                    const uint64_t *tile_off, uint64_t *counts) {
    __shared__ uint32_t sa[kTile];
    __shared__ uint32_t sb[kTile + 1];
    __shared__ uint64_t bounds[2];
    __shared__ uint32_t red[kThreads / 32];
    const uint64_t total = tile_off[npairs];
    for (uint64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const uint32_t p = tile_pair(tile_off, npairs, tile);
        const uint64_t t = tile - tile_off[p];
        const PairPlan pl = plan[p];
        lh_set a = A[p], b = B[p];
        if (pl.swap) { lh_set x = a; a = b; b = x; }
        uint32_t cnt = 0;
        if (pl.kind == K_MERGE) {
            const uint64_t nd = a.n + b.n;
            const uint64_t d0 = t * kTile, d1 = min(nd, d0 + kTile);
            if (threadIdx.x == 0) bounds[0] = mp_split(a.data, a.n, b.data, b.n, d0);
            else if (threadIdx.x == 32) bounds[1] = mp_split(a.data, a.n, b.data, b.n, d1);
            __syncthreads();
            const uint64_t i0 = bounds[0], i1 = bounds[1];
            const uint64_t j0 = d0 - i0, j1 = d1 - i1;
            const uint32_t la = (uint32_t)(i1 - i0), lb = (uint32_t)(j1 - j0);
            const bool has_ext = j1 < b.n;
            const uint32_t lbx = lb + (has_ext ? 1u : 0u);
            // all loads of this thread in flight before any shared store
            uint32_t ra[kItems], rb[kItems + 1];
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                const uint32_t k = threadIdx.x + r * kThreads;
                ra[r] = k < la ? __ldg(a.data + i0 + k) : 0u;
                rb[r] = k < lbx ? __ldg(b.data + j0 + k) : 0u;
            }
            rb[kItems] = (threadIdx.x == 0 && kTile < lbx) ? __ldg(b.data + j0 + kTile) : 0u;
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                const uint32_t k = threadIdx.x + r * kThreads;
                if (k < la) sa[k] = ra[r];
                if (k < lbx) sb[k] = rb[r];
            }
            if (threadIdx.x == 0 && kTile < lbx) sb[kTile] = rb[kItems];
            __syncthreads();
            const uint32_t s = threadIdx.x * kItems;
            const uint32_t e = min(s + kItems, la + lb);
            if (s < e) {
                uint32_t ii = sm_split(sa, la, sb, lb, s);
                uint32_t jj = s - ii;
                for (uint32_t step = s; step < e; ++step) {
                    if (ii < la && (jj >= lb || sa[ii] <= sb[jj])) {
                        uint32_t av = sa[ii];
                        bool head = jj < lb || (jj == lb && has_ext);
                        if (head && sb[jj] == av) ++cnt;
                        ++ii;
                    } else {
                        ++jj;
                    }
                }
            }
        } else if (pl.kind == K_PROBE) {
            const uint64_t base = t * kTile;
            uint32_t x[kItems];
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                const uint64_t i = base + threadIdx.x + r * kThreads;
                x[r] = i < a.n ? __ldg(a.data + i) : 0u;
            }
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                const uint64_t i = base + threadIdx.x + r * kThreads;
                if (i >= a.n) continue;
                uint64_t l = 0, h = b.n;
                while (l < h) {
                    uint64_t m = (l + h) >> 1;
                    if (__ldg(b.data + m) < x[r]) l = m + 1;
                    else h = m;
                }
                cnt += (l < b.n && __ldg(b.data + l) == x[r]) ? 1u : 0u;
            }
        } else if (pl.kind == K_UBS) {
            const uint64_t base = t * kTile;
            uint32_t x[kItems];
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                const uint64_t i = base + threadIdx.x + r * kThreads;
                x[r] = i < a.n ? __ldg(a.data + i) : b.base - 1u;  // padding: below the base when base > 0
            }
            uint32_t w[kItems];
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                const uint64_t i = base + threadIdx.x + r * kThreads;
                const uint32_t d = x[r] - b.base;
                const bool in = i < a.n && x[r] >= b.base && (uint64_t)(d >> 5) < b.n;
                w[r] = in ? __ldg(b.data + (d >> 5)) : 0u;
            }
#pragma unroll
            for (int r = 0; r < kItems; ++r) cnt += (w[r] >> ((x[r] - b.base) & 31u)) & 1u;
        } else if (pl.kind == K_BB) {
            // word ranges start on 128-bit boundaries (bases are multiples of
            // 128 values = 4 words), so uint4 loads are aligned
            const uint64_t w0 = pl.lo_w + t * kTile, w1 = min(pl.hi_w, w0 + kTile);
            const uint4 *pa = (const uint4 *)(a.data + (w0 - (a.base >> 5)));
            const uint4 *pb = (const uint4 *)(b.data + (w0 - (b.base >> 5)));
            const uint32_t nv = (uint32_t)((w1 - w0) >> 2);
            for (uint32_t k = threadIdx.x; k < nv; k += kThreads) {
                uint4 x = __ldg(pa + k), y = __ldg(pb + k);
                cnt += __popc(x.x & y.x) + __popc(x.y & y.y) + __popc(x.z & y.z) + __popc(x.w & y.w);
            }
        }
        uint32_t tot = block_sum(cnt, red);
        if (threadIdx.x == 0 && tot) atomicAdd((unsigned long long *)(counts + p), (unsigned long long)tot);
        __syncthreads();
    }
}

// ---- descriptor-driven variant (allocating entry point) ---------------------
// Everything a tile needs -- its pair, slice pointers and lengths -- is
// computed for all tiles at once by k_isect_tiles, so a CTA's only dependent
// load per tile is its 48-byte descriptor, and the next tile's data loads are
// issued into registers before the current tile is merged.

struct __align__(16) TileDesc {
    const uint32_t *a;   // merge: A slice; probe / ubs: uint elements; bs: A words
    const uint32_t *b;   // merge: B slice; probe: B set; ubs: B words; bs: B words
    uint32_t la, lb;     // merge: slice lengths; probe / ubs: elements; bs: words
    uint32_t pair, kind; // kind | 256 when the merge slice of B has one extra head element
    uint64_t bn;         // probe: |B|; ubs: B words
    uint32_t bbase;      // ubs: B base value
    uint32_t room;       // merge: elements after each slice that stay inside
                         // its array (A: bits 0-1, B: bits 2-3, at most 3);
                         // bit 4: both arrays 16-byte aligned
};

__global__ void k_isect_tiles(uint32_t npairs, const lh_set *A, const lh_set *B, const PairPlan *plan,
                              const uint64_t *tile_off, TileDesc *desc) {
    const uint64_t total = tile_off[npairs];
    for (uint64_t tile = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; tile < total;
         tile += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = tile_pair(tile_off, npairs, tile);
        const uint64_t t = tile - tile_off[p];
        const PairPlan pl = plan[p];
        lh_set a = A[p], b = B[p];
        if (pl.swap) { lh_set x = a; a = b; b = x; }
        TileDesc d;
        d.pair = p;
        d.kind = pl.kind;
        d.bn = 0;
        d.bbase = 0;
        d.room = 0;
        if (pl.kind == K_MERGE) {
            const uint64_t nd = a.n + b.n;
            const uint64_t d0 = t * kTile, d1 = min(nd, d0 + kTile);
            const uint64_t i0 = mp_split(a.data, a.n, b.data, b.n, d0);
            const uint64_t i1 = mp_split(a.data, a.n, b.data, b.n, d1);
            const uint64_t j0 = d0 - i0, j1 = d1 - i1;
            d.a = a.data + i0;
            d.b = b.data + j0;
            d.la = (uint32_t)(i1 - i0);
            d.lb = (uint32_t)(j1 - j0);
            if (j1 < b.n) d.kind |= 256u;
            const uint64_t bend = j1 + (j1 < b.n ? 1 : 0);
            d.room = (uint32_t)min((uint64_t)3, a.n - i1) | ((uint32_t)min((uint64_t)3, b.n - bend) << 2);
            if (((uintptr_t)a.data & 15u) == 0 && ((uintptr_t)b.data & 15u) == 0) d.room |= 16u;
        } else if (pl.kind == K_BB) {
            const uint64_t w0 = pl.lo_w + t * kTile, w1 = min(pl.hi_w, w0 + kTile);
            d.a = a.data + (w0 - (a.base >> 5));
            d.b = b.data + (w0 - (b.base >> 5));
            d.la = d.lb = (uint32_t)(w1 - w0);
        } else {  // probe or uint cap bs: a tile of the uint side
            const uint64_t i0 = t * kTile;
            d.a = a.data + i0;
            d.la = (uint32_t)min((uint64_t)kTile, a.n - i0);
            d.b = b.data;
            d.lb = 0;
            d.bn = b.n;
            d.bbase = b.base;
        }
        desc[tile] = d;
    }
}

// ---- TMA-staged merge tiles ------------------------------------------------
// Merge slices are staged by cp.async.bulk (one copy per slice, issued by one
// thread, completion on an mbarrier) into two shared buffers: the next tile's
// slices load while the current one is merged.  A copy must start and end on
// 16-byte boundaries, so it covers the slice rounded out to whole 16-byte
// words where the array allows it; elements the rounded copy cannot cover
// (a slice end closer than 16 bytes to its array's end) are fetched with
// plain loads.  Descriptors are read two tiles ahead.  Waits are bounded.

constexpr uint32_t kBufA = kTile + 8, kBufB = kTile + 16;
constexpr uint32_t kWaitLimit = 1u << 22;
// Bound of the second wait after a timeout: copies already issued may still
// land, so the block polls their phase this much longer before it exits.
constexpr uint32_t kDrainLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init1(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arm(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Copy window of a slice [p, p + len) whose array has `room` readable
// elements after the slice: the 16-byte words from the one holding p up to
// the end rounded up (or down, when rounding up would leave the array), as
// element offsets [lo, hi) relative to p (lo in -3..0; no window when hi <= lo
// or the arrays are not 16-byte aligned).
__device__ __forceinline__ void copy_window(const uint32_t *p, uint32_t len, uint32_t room, bool aligned, int &lo,
                                            int &hi) {
    lo = hi = 0;
    if (!aligned) return;
    const int64_t a = (int64_t)(((uintptr_t)p) >> 2);
    const int64_t start = a & ~3ll, end = a + len;
    const int64_t up = (end + 3) & ~3ll;
    const int64_t stop = (up - end <= (int64_t)room) ? up : (end & ~3ll);
    lo = (int)(start - a);
    hi = (int)(stop - a);
    if (hi < lo) hi = lo;
}

// Issue the staging of merge tile d into buffers (sa, sb): thread 0 arms the
// barrier and starts the bulk copies; every thread plain-loads its share of
// the elements the copies leave out.  Returns the buffer offsets of element 0.
__device__ __forceinline__ void stage_merge(const TileDesc &d, uint32_t *sa, uint32_t *sb, uint64_t *bar, int &offa,
                                            int &offb) {
    const bool aligned = (d.room >> 4) & 1u;
    const uint32_t lbx = d.lb + ((d.kind >> 8) & 1u);
    int alo, ahi, blo, bhi;
    copy_window(d.a, d.la, d.room & 3u, aligned, alo, ahi);
    copy_window(d.b, lbx, (d.room >> 2) & 3u, aligned, blo, bhi);
    offa = -alo;
    offb = -blo;
    const uint32_t na = (uint32_t)(ahi - alo), nb = (uint32_t)(bhi - blo);
    if (threadIdx.x == 0) {
        // earlier generic-proxy reads of this buffer come before the async copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arm(bar, 4u * (na + nb));
        if (na) bulk_g2s(sa, d.a + alo, 4u * na, bar);
        if (nb) bulk_g2s(sb, d.b + blo, 4u * nb, bar);
    }
    // elements past the copy windows
    const uint32_t a_from = na ? (uint32_t)max(ahi, 0) : 0u, b_from = nb ? (uint32_t)max(bhi, 0) : 0u;
    for (uint32_t k = a_from + threadIdx.x; k < d.la; k += kThreads) sa[offa + k] = __ldg(d.a + k);
    for (uint32_t k = b_from + threadIdx.x; k < lbx; k += kThreads) sb[offb + k] = __ldg(d.b + k);
}

// ---- merge tiles, version 4 --------------------------------------------------
// One linear staging buffer filled by cp.async.bulk (the next tile's copies
// overlap the current merge) and one padded copy of the current tile
// (index i stored at i + i/32) so that threads whose merge ranges start 8
// words apart hit distinct banks.  Sentinels (0xFFFFFFFF) close both padded
// slices, so the branch-free merge needs no bounds tests; pairs whose sets
// hold that value use the probe path instead (k_plan).

constexpr uint32_t kSwz = kTile + 2 + (kTile + 2) / 32 + 2;
__device__ __forceinline__ uint32_t swz(uint32_t i) { return i + (i >> 5); }

// merge-path split on the padded slices (ties: A first)
__device__ __forceinline__ uint32_t sw_split(const uint32_t *a, uint32_t na, const uint32_t *b, uint32_t nb,
                                             uint32_t d) {
    uint32_t lo = d > nb ? d - nb : 0, hi = min(d, na);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const bool right = a[swz(mid)] <= b[swz(d - mid - 1)];
        lo = right ? mid + 1 : lo;
        hi = right ? hi : mid;
    }
    return lo;
}

// Merge tiles only: the probe, uint-cap-bs and bs-cap-bs tiles of a batch
// are counted by k_isect_lean (launched beside this kernel) and skipped here.
__global__ void __launch_bounds__(kThreads) k_isect4(const TileDesc *desc, uint64_t total, uint64_t *counts,
                                                     uint32_t *status) {
    __shared__ __align__(128) uint32_t la_buf[kBufA];
    __shared__ __align__(128) uint32_t lb_buf[kBufB];
    __shared__ uint32_t pa[kSwz];
    __shared__ uint32_t pb[kSwz];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t red[kThreads / 32];
    uint64_t tile = blockIdx.x;
    if (tile >= total) return;
    if (threadIdx.x == 0) {
        mbar_init1(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t uses = 0;
    int offa = 0, offb = 0;
    TileDesc d = desc[tile];
    TileDesc dn = d;
    if (tile + gridDim.x < total) dn = desc[tile + gridDim.x];
    if ((d.kind & 255u) == K_MERGE) {
        stage_merge(d, la_buf, lb_buf, &bar, offa, offb);
        uses++;
    }
    while (tile < total) {
        const uint64_t next = tile + gridDim.x;
        TileDesc dnn = dn;
        if (next + gridDim.x < total) dnn = desc[next + gridDim.x];
        const uint32_t kind = d.kind & 255u;
        const uint32_t la = d.la, lb = d.lb;
        const uint32_t lbx = lb + ((d.kind >> 8) & 1u);
        bool waited = true;
        if (kind == K_MERGE) waited = mbar_wait_bounded(&bar, (uses - 1) & 1u);
        if (__syncthreads_or(!waited)) {
            // the bulk copies of this tile may still land in shared memory:
            // no new copy is issued, and thread 0 keeps polling the same
            // phase with a much longer bound before the block may exit
            if (threadIdx.x == 0) {
                lh_set_status(status, LH_ETIMEOUT);
                mbar_wait_bounded(&bar, (uses - 1) & 1u, kDrainLimit);
            }
            __syncthreads();
            return;
        }
        if (kind == K_MERGE) {
            // linear staging -> padded copy with sentinels
            for (uint32_t k = threadIdx.x; k < la; k += kThreads) pa[swz(k)] = la_buf[offa + k];
            for (uint32_t k = threadIdx.x; k < lbx; k += kThreads) pb[swz(k)] = lb_buf[offb + k];
            if (threadIdx.x == 0) {
                pa[swz(la)] = 0xFFFFFFFFu;
                pb[swz(lbx)] = 0xFFFFFFFFu;
            }
        }
        __syncthreads();
        // the staging buffer is free: start the next merge tile's copies
        if (next < total && (dn.kind & 255u) == K_MERGE) {
            stage_merge(dn, la_buf, lb_buf, &bar, offa, offb);
            uses++;
        }
        uint32_t cnt = 0;
        if (kind == K_MERGE) {
            const uint32_t s = threadIdx.x * kItems;
            const uint32_t e = min(s + kItems, la + lb);
            if (s < e) {
                uint32_t ii = sw_split(pa, la, pb, lb, s);
                uint32_t jj = s - ii;
                uint32_t a = pa[swz(ii)], b = pb[swz(jj)];
#pragma unroll
                for (int k = 0; k < kItems; ++k) {
                    if (s + k < e) {
                        const bool ta = a <= b;
                        cnt += (a == b) ? 1u : 0u;  // a consumed while the B head equals it
                        if (ta) a = pa[swz(++ii)];
                        else b = pb[swz(++jj)];
                    }
                }
            }
        }
        const uint32_t tot = block_sum(cnt, red);  // ends with a barrier: the padded tile is free again
        if (threadIdx.x == 0 && tot) atomicAdd((unsigned long long *)(counts + d.pair), (unsigned long long)tot);
        tile = next;
        d = dn;
        dn = dnn;
    }
    // every staged tile was consumed (a tile is staged only when a later
    // iteration exists to wait for it), so no copy is in flight here
}

// Probe, uint-cap-bs and bs-cap-bs tiles need no shared staging, so they run
// in a kernel of their own whose occupancy is not held down by the merge
// tiles' shared buffers: more tiles per SM keep more loads in flight (the
// bs-cap-bs batches are bound by loads in flight).  Tiles of other kinds are
// skipped (k_isect4 counts the merge tiles).
constexpr int kLeanCtas = 6;

__global__ void __launch_bounds__(kThreads, kLeanCtas) k_isect_lean(const TileDesc *desc, uint64_t total,
                                                                    uint64_t *counts) {
    __shared__ uint32_t red[kThreads / 32];
    for (uint64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const TileDesc d = desc[tile];
        const uint32_t kind = d.kind & 255u;
        if (kind != K_UBS && kind != K_PROBE && kind != K_BB) continue;  // the same for the whole block
        const uint32_t la = d.la;
        uint32_t cnt = 0;
        if (kind == K_BB) {
            const uint4 *qa = (const uint4 *)d.a;
            const uint4 *qb = (const uint4 *)d.b;
            const uint32_t nv = la >> 2;
            constexpr int kVec = kTile / 4 / kThreads;
            uint4 xa[kVec], xb[kVec];
#pragma unroll
            for (int u = 0; u < kVec; ++u) {
                const uint32_t k = threadIdx.x + u * kThreads;
                xa[u] = k < nv ? __ldg(qa + k) : make_uint4(0, 0, 0, 0);
                xb[u] = k < nv ? __ldg(qb + k) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < kVec; ++u)
                cnt += __popc(xa[u].x & xb[u].x) + __popc(xa[u].y & xb[u].y) + __popc(xa[u].z & xb[u].z) +
                       __popc(xa[u].w & xb[u].w);
        } else {
            uint32_t x[kItems];
#pragma unroll
            for (int r = 0; r < kItems; ++r) {
                const uint32_t k = threadIdx.x + r * kThreads;
                x[r] = k < la ? __ldg(d.a + k) : 0u;
            }
            if (kind == K_UBS) {
                uint32_t w[kItems];
#pragma unroll
                for (int r = 0; r < kItems; ++r) {
                    const uint32_t k = threadIdx.x + r * kThreads;
                    const uint32_t dd = x[r] - d.bbase;
                    const bool in = k < la && x[r] >= d.bbase && (uint64_t)(dd >> 5) < d.bn;
                    w[r] = in ? __ldg(d.b + (dd >> 5)) : 0u;
                }
#pragma unroll
                for (int r = 0; r < kItems; ++r) cnt += (w[r] >> ((x[r] - d.bbase) & 31u)) & 1u;
            } else {
#pragma unroll
                for (int r = 0; r < kItems; ++r) {
                    const uint32_t k = threadIdx.x + r * kThreads;
                    if (k >= la) continue;
                    uint64_t l = 0, h = d.bn;
                    while (l < h) {
                        const uint64_t m = (l + h) >> 1;
                        if (__ldg(d.b + m) < x[r]) l = m + 1;
                        else h = m;
                    }
                    cnt += (l < d.bn && __ldg(d.b + l) == x[r]) ? 1u : 0u;
                }
            }
        }
        const uint32_t tot = block_sum(cnt, red);
        if (threadIdx.x == 0 && tot) atomicAdd((unsigned long long *)(counts + d.pair), (unsigned long long)tot);
    }
}

}  // namespace

extern "C" lh_status lh_intersect_count_batch(lh_ctx *ctx, uint32_t npairs, const lh_set *a,
                                              const lh_set *b, uint64_t *counts) {
    if (!ctx) return LH_EINVAL;
    if (npairs == 0) return LH_OK;
    if (!a || !b || !counts) return lh_fail(ctx, LH_EINVAL, "null argument");
    PairPlan *plan = nullptr;
    uint64_t *tiles = nullptr, *off = nullptr;
    uint64_t ntiles = 0;
    // off[npairs]: the tile total; off[npairs + 1]: the merge tiles among them
    lh_status s = lh_alloc(ctx, &plan, npairs);
    if (s == LH_OK) s = lh_alloc(ctx, &tiles, npairs);
    if (s == LH_OK) s = lh_alloc(ctx, &off, (size_t)npairs + 2);
    if (s == LH_OK) {
        cudaMemsetAsync(counts, 0, npairs * sizeof(uint64_t), ctx->stream);
        cudaMemsetAsync(off + npairs + 1, 0, sizeof(uint64_t), ctx->stream);
        LH_TRACED(ctx, "k_plan", k_plan<<<lh_blocks(npairs, 256), 256, 0, ctx->stream>>>(
                                     npairs, a, b, plan, tiles, (unsigned long long *)(off + npairs + 1)));
        s = lh_scan_u64_to_u64(ctx, tiles, off, npairs);
    }
    uint64_t rb[2] = {0, 0};
    if (s == LH_OK) s = lh_readback(ctx, off + npairs, sizeof(rb), rb);
    ntiles = rb[0];
    const uint64_t n_merge = rb[1];
    TileDesc *desc = nullptr;
    if (s == LH_OK) s = lh_alloc(ctx, &desc, ntiles);
    if (s == LH_OK && ntiles) {
        LH_TRACED(ctx, "k_isect_tiles", k_isect_tiles<<<lh_blocks(ntiles, 256, (unsigned)ctx->num_sms * 8), 256, 0, ctx->stream>>>(
                                            npairs, a, b, plan, off, desc));
        // merge tiles in k_isect4 (shared staging), the other kinds in
        // k_isect_lean; a batch of one kind launches one kernel
        const bool lean = n_merge < ntiles;
        if (n_merge) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_isect4, kThreads, 0);
            if (per_sm < 1) per_sm = 1;
            const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)ctx->num_sms * per_sm);
            LH_TRACED(ctx, "k_isect", k_isect4<<<grid, kThreads, 0, ctx->stream>>>(desc, ntiles, counts, ctx->d_status));
        }
        if (lean) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_isect_lean, kThreads, 0);
            if (per_sm < 1) per_sm = 1;
            const unsigned grid = (unsigned)std::min<uint64_t>(ntiles - n_merge, (uint64_t)ctx->num_sms * per_sm);
            LH_TRACED(ctx, "k_isect_lean", k_isect_lean<<<grid, kThreads, 0, ctx->stream>>>(desc, ntiles, counts));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "intersect: %s", cudaGetErrorString(e));
    }
    lh_free(ctx, plan);
    lh_free(ctx, tiles);
    lh_free(ctx, off);
    lh_free(ctx, desc);
    return s;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of lh_intersect_count_batch.
//
// Some callers cannot allocate device memory on their query path: a host
// application whose buffer pool or framework allocator owns all of the
// GPU's memory, or a latency-bound loop where an allocation could stall or
// fail.  This entry point keeps its per-pair scratch (layout plan, tile
// count, tile offset) in one file-scope device array instead of calling the
// allocator.  The array holds kNoAllocMaxPairs pairs (about 2.6 MB) and stays
// resident on every GPU that loads this library until the process exits.
// All calls share it: calls whose work overlaps on the GPU (different
// streams, or different contexts on one device) race on it.

namespace {

constexpr uint32_t kNoAllocMaxPairs = 65536;
constexpr size_t kNaPlanBytes = sizeof(PairPlan) * kNoAllocMaxPairs;
constexpr size_t kNaTilesBytes = sizeof(uint64_t) * kNoAllocMaxPairs;
constexpr size_t kNaOffBytes = sizeof(uint64_t) * (kNoAllocMaxPairs + 1);
constexpr size_t kNaPlanAt = 0;
constexpr size_t kNaTilesAt = (kNaPlanAt + kNaPlanBytes + 255) & ~size_t(255);
constexpr size_t kNaOffAt = (kNaTilesAt + kNaTilesBytes + 255) & ~size_t(255);
constexpr size_t kNaBytes = kNaOffAt + kNaOffBytes;

static __device__ __align__(256) unsigned char g_isect_scratch[kNaBytes];

// Exclusive scan of n <= kNoAllocMaxPairs tile counts by one block of 1024
// threads (the allocating path's multi-block scan needs temporaries).
__global__ void __launch_bounds__(1024) k_scan_one_block(const uint64_t *in, uint32_t n, uint64_t *out) {
    __shared__ uint64_t warp_tot[32];
    __shared__ uint64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t v = i < n ? in[i] : 0;
        uint64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t t = __shfl_up_sync(LH_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint64_t w = warp_tot[lane], wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint64_t t = __shfl_up_sync(LH_FULL, wi, o);
                if (lane >= o) wi += t;
            }
            warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
        }
        __syncthreads();
        if (i < n) out[i] = carry + warp_tot[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += warp_tot[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

std::mutex g_na_mu;
constexpr int kNaMaxDevices = 64;
unsigned char *g_na_ptr[kNaMaxDevices] = {nullptr};

// Device address of the scratch array on the context's device, looked up
// once per device with that device current.
lh_status noalloc_scratch(lh_ctx *ctx, unsigned char **out) {
    int cur = -1;
    LH_CU(cudaGetDevice(&cur));
    if (cur != ctx->device)
        return lh_fail(ctx, LH_EINVAL, "the context's device (%d) is not the current device (%d)", ctx->device, cur);
    if (cur < 0 || cur >= kNaMaxDevices) return lh_fail(ctx, LH_EUNSUPPORTED, "device index %d", cur);
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[cur]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_isect_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return lh_fail(ctx, LH_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        }
        g_na_ptr[cur] = (unsigned char *)p;
    }
    *out = g_na_ptr[cur];
    return LH_OK;
}

}  // namespace

extern "C" lh_status lh_intersect_count_batch_noalloc(lh_ctx *ctx, uint32_t npairs, const lh_set *a,
                                                      const lh_set *b, uint64_t *counts) {
    if (!ctx) return LH_EINVAL;
    if (npairs > kNoAllocMaxPairs)
        return lh_fail(ctx, LH_EINVAL, "npairs %u exceeds the allocation-free limit of %u pairs", npairs,
                       kNoAllocMaxPairs);
    if (npairs == 0) return LH_OK;
    if (!a || !b || !counts) return lh_fail(ctx, LH_EINVAL, "null argument");
    unsigned char *scratch = nullptr;
    LH_TRY(noalloc_scratch(ctx, &scratch));
    PairPlan *plan = (PairPlan *)(scratch + kNaPlanAt);
    uint64_t *tiles = (uint64_t *)(scratch + kNaTilesAt);
    uint64_t *off = (uint64_t *)(scratch + kNaOffAt);
    // counts start at zero: k_isect adds into them; plan, tiles and off are
    // fully rewritten below for the first npairs pairs
    LH_CU(cudaMemsetAsync(counts, 0, npairs * sizeof(uint64_t), ctx->stream));
    LH_TRACED(ctx, "k_plan", k_plan<<<lh_blocks(npairs, 256), 256, 0, ctx->stream>>>(npairs, a, b, plan, tiles));
    LH_TRACED(ctx, "k_scan_one_block", k_scan_one_block<<<1, 1024, 0, ctx->stream>>>(tiles, npairs, off));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_isect, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    unsigned grid = (unsigned)(ctx->num_sms * per_sm);
    LH_TRACED(ctx, "k_isect", k_isect<<<grid, kThreads, 0, ctx->stream>>>(npairs, a, b, plan, off, counts));
    LH_LAUNCH_CHECK();
    return LH_OK;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded device waits: one warp waits on an mbarrier that
// nothing will ever arrive at, gives up after `spins` tries, and records
// LH_ETIMEOUT in the context's status word -- the path every TMA / mbarrier
// wait of this library takes when a copy never lands.  No fault, no trap.
namespace {
__global__ void k_selftest_wait(uint32_t spins, uint32_t *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init1(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool done = false;
    for (uint32_t i = 0; i < spins && !done; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(&bar))
            : "memory");
        done = ok != 0;
    }
    if (__syncthreads_or(!done) && threadIdx.x == 0) lh_set_status(status, LH_ETIMEOUT);
}
}  // namespace

extern "C" lh_status lh_selftest_bounded_wait(lh_ctx *ctx, uint32_t spins) {
    if (!ctx) return LH_EINVAL;
    if (spins == 0 || spins > (1u << 20)) return lh_fail(ctx, LH_EINVAL, "spins must be 1..2^20");
    LH_TRACED(ctx, "k_selftest_wait", k_selftest_wait<<<1, 32, 0, ctx->stream>>>(spins, ctx->d_status));
    LH_LAUNCH_CHECK();
    return lh_sync(ctx);
}
