// Generic worst-case-optimal join-aggregate driver (Algorithm 1, Section 2.4)
// with AJAR aggregation (Section 2.3) and GROUP BY on annotations or keys
// (Section 5).
//
// Algorithm 1 recurses one attribute at a time; on the GPU the recursion is
// unrolled breadth-first in bounded chunks.  The frontier at depth d holds,
// for every bound prefix tuple, each relation's position in its trie.  For
// depth d (attribute v = order[d]):
//   1. sizes:  per frontier entry, the candidate set of every relation that
//      contains v (its level-0 set, or the children of its bound parent); the
//      smallest one drives.
//   2. scan:   exclusive prefix of driver sizes = a flat candidate space, so
//      that one thread handles one candidate whatever the skew of set sizes.
//   3. expand: each candidate x of the driver is probed in every other set
//      (bitset: one word and a rank; uint: binary search) -- the k-way
//      intersection; survivors become the next frontier (warp-aggregated
//      compaction), or at the last attribute are counted / aggregated.
// At the root (depth 0) the sets are level-0 sets whose sizes the host
// already knows, so step 1 and the scan are skipped there.
// The candidate space is cut into chunks of at most `cap` candidates, so the
// frontier memory is bounded whatever the output size; each chunk recurses
// before the next is expanded (depth-first over chunks).  A chunk of at most
// kPadFrontierMax candidates hands its survivor count to the next depth on
// the device (that depth runs over the chunk's capacity, padding sized 0),
// so the host reads back one candidate total per depth.
#include <chrono>
#include <cmath>

#include "lh_join.cuh"

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kSmemGroupsMax = 1024;
constexpr uint64_t kLastChunk = 1ull << 28;   // candidates per last-attribute launch
constexpr uint32_t kPadFrontierMax = 1u << 18;  // chunks up to this size pass their survivor count on the device
constexpr int kMaxG = LH_MAX_GROUP;
constexpr uint32_t kPrivSlots = 256;                 // per-warp private GROUP BY table
constexpr unsigned long long kPrivEmpty = ~0ull;
constexpr uint32_t kHashSpin = 1u << 20;             // bound of a wait on a slot being written

enum { M_EMIT = 0, M_COUNT = 1, M_AGG = 2 };
enum { G_DENSE = 0, G_PRIVATE = 1, G_SHARED = 2 };

// Shared GROUP BY table (Section 5, the concurrent hash map): open
// addressing over `cap` slots (a power of two).  tag 0 = empty; an even tag
// (hash with the low bit clear) = claimed, key still being written; an odd
// tag (the tuple's hash, low bit set) = key visible.  keys: ncol x cap,
// column-major.
struct HTab {
    unsigned long long *tag;
    uint32_t *keys;
    double *sum;
    unsigned long long *cnt;
    uint32_t cap;
};

struct JEdge {
    DTrie t;
    const float *flat;
    uint32_t flat_n;
    uint32_t is_flat;
    uint32_t anno_kind;  // 0 none, 1 f32, 2 compensated pair
    const float *a_hi;
    const float *a_lo;
};

struct JDepth {
    uint32_t np;
    uint8_t e[LH_MAX_EDGES];
    uint8_t lvl[LH_MAX_EDGES];
};

struct JQuery {
    JEdge E[LH_MAX_EDGES];
    uint32_t ne;
    JDepth D[LH_MAX_ATTRS];
    uint32_t nd;
    uint32_t ngc;                 // group columns
    uint32_t g_is_key[kMaxG];     // 1: key attribute value, 0: int32 annotation column
    uint32_t g_edge[kMaxG];
    const int32_t *g_col[kMaxG];
    uint32_t g_depth[kMaxG];      // depth that binds the key attribute
    uint32_t g_slot[kMaxG];       // frontier slot of a key group value
    uint32_t g_card[kMaxG];       // 0 = undeclared domain (hash modes only)
    uint32_t g_shift[kMaxG];      // private tables: bit offset of the column in the packed key
    uint32_t ngroups;             // dense mode: groups (1 when no GROUP BY)
    uint32_t gmode;               // G_DENSE, G_PRIVATE or G_SHARED
    HTab ht;
    uint32_t count_only;          // COUNT semiring: no annotation product
};

// 64-bit finalizer of splitmix64 (Steele, Lea and Flood, 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// hash of a key tuple, odd (the ready tag of its slot)
__device__ __forceinline__ unsigned long long tuple_hash(const uint32_t *kv, uint32_t n) {
    unsigned long long h = 0x243f6a8885a308d3ull;
    for (uint32_t k = 0; k < n; ++k) h = mix64(h ^ ((unsigned long long)kv[k] + ((unsigned long long)k << 32)));
    return h | 1ull;
}

// Adds (v, c) to the group of key tuple kv in the shared table; false (and
// the status word set) when the table is full or a slot stays claimed.
__device__ bool ht_upsert(const HTab &H, uint32_t ncol, const uint32_t *kv, double v, unsigned long long c,
                          uint32_t *status) {
    const unsigned long long h = tuple_hash(kv, ncol), claimed = h & ~1ull;
    uint32_t slot = (uint32_t)(h >> 20) & (H.cap - 1);
    volatile unsigned long long *vtag = H.tag;
    volatile uint32_t *vkeys = H.keys;
    for (uint32_t probe = 0; probe < H.cap; ++probe) {
        unsigned long long t = vtag[slot];
        if (t == 0) {
            const unsigned long long prev = atomicCAS(H.tag + slot, 0ull, claimed);
            if (prev == 0) {
                for (uint32_t k = 0; k < ncol; ++k) H.keys[(size_t)k * H.cap + slot] = kv[k];
                __threadfence();
                atomicExch(H.tag + slot, h);
                atomicAdd(H.sum + slot, v);
                atomicAdd(H.cnt + slot, c);
                return true;
            }
            t = prev;
        }
        if ((t | 1ull) == h) {
            for (uint32_t spin = 0; (t & 1ull) == 0; ++spin) {
                if (spin >= kHashSpin) {
                    lh_set_status(status, LH_ETIMEOUT);
                    return false;
                }
                t = vtag[slot];
            }
            __threadfence();
            bool eq = true;
            for (uint32_t k = 0; k < ncol; ++k) eq = eq && vkeys[(size_t)k * H.cap + slot] == kv[k];
            if (eq) {
                atomicAdd(H.sum + slot, v);
                atomicAdd(H.cnt + slot, c);
                return true;
            }
        }
        slot = (slot + 1) & (H.cap - 1);
    }
    lh_set_status(status, LH_EOVERFLOW);
    return false;
}

__device__ __forceinline__ void unpack_key(const JQuery &q, unsigned long long K, uint32_t *kv) {
    for (uint32_t k = 0; k < q.ngc; ++k) {
        const uint32_t bits = (k + 1 < q.ngc ? q.g_shift[k + 1] : 64u) - q.g_shift[k];
        const unsigned long long m = bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
        kv[k] = (uint32_t)((K >> q.g_shift[k]) & m);
    }
}

// Set slot flags and compaction of the shared table (at the wait).
__global__ void k_ht_flags(const unsigned long long *tag, uint32_t cap, uint32_t *flag) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x)
        flag[i] = (tag[i] & 1ull) ? 1u : 0u;
}
__global__ void k_ht_scatter(HTab H, uint32_t ncol, const uint64_t *pos, uint64_t G, uint32_t *keys, double *sum,
                             uint64_t *cnt) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < H.cap; i += gridDim.x * blockDim.x) {
        if (!(H.tag[i] & 1ull)) continue;
        const uint64_t g = pos[i];
        for (uint32_t k = 0; k < ncol; ++k) keys[(size_t)k * G + g] = H.keys[(size_t)k * H.cap + i];
        sum[g] = H.sum[i];
        cnt[g] = H.cnt[i];
    }
}

__device__ __forceinline__ uint32_t find_entry(const uint64_t *off, uint32_t nF, uint64_t c, uint32_t lo = 0) {
    uint32_t hi = nF;  // off[lo] <= c < off[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Frontier entries of one block-iteration of candidates: the block's first
// and last candidates are located once in the global offsets, the offsets
// in between are staged in shared memory, and every thread finds its entry
// there (a few shared loads instead of a search over the whole frontier).
constexpr uint32_t kWin = 256;

// ---- count-only intersection of two sets at the last attribute ------------
// A COUNT join without GROUP BY needs only |S ∩ T| at its last attribute.
// Frontier entries whose smaller set holds at least kWarpMinSet elements are
// taken off the per-candidate path and counted by warps, in work items of at
// most kSegWork elements, so a hub entry is spread over many warps:
//   MERGE   both sets uint, |T| <= kMergeRatio |S|: merge path.  Item g covers
//           diagonals [g kSegWork, (g+1) kSegWork) of the merge of S and T;
//           the warp steps through it with a 32-element window of each set,
//           finds every S element's lower bound in T's window with five
//           shuffles, counts the equal ones below the windows' common bound
//           with a ballot, and advances each window past that bound.
//   SCAN_S  T a bitset, or T much larger than S: lanes take S's elements,
//           each probes T (bitset word, or a binary search whose lower end
//           moves forward with the warp's previous element -- S is sorted).
//   SCAN_T  S a bitset and T uint of comparable size: lanes take T's
//           elements and probe S's bitset.
constexpr uint32_t kWarpMinSet = 32;
constexpr uint32_t kSegWork = 2048;
constexpr uint32_t kMergeRatio = 8;
constexpr unsigned long long kNoItem = ~0ull;
enum { K_MERGE = 0, K_SCAN_S = 1, K_SCAN_T = 2 };

struct LastPair {
    uint32_t pS, pT;            // positions (in the depth's relation list) of the smaller and the other set
    uint32_t sLo, sHi, tLo, tHi, sSet, tSet;
    uint32_t kind;
    uint64_t work, nseg;
};

// The two sets of frontier entry i at the last depth (both relations stored
// as tries), the smaller one first on ties as k_sizes picks its driver.
__device__ __forceinline__ void pair_side(const JQuery &q, const JDepth &D, const uint32_t *posF, uint32_t capF,
                                          uint32_t i, uint32_t p, uint32_t &lo, uint32_t &hi, uint32_t &set,
                                          bool &bs) {
    const JEdge &E = q.E[D.e[p]];
    const uint32_t L = D.lvl[p];
    const uint32_t parent = L ? posF[(uint64_t)D.e[p] * capF + i] : 0u;
    lh_set_range(E.t, L, parent, lo, hi);
    set = L ? parent : 0u;
    const DLevel &lv = E.t.lv[L];
    bs = lv.bs_slot != nullptr && __ldg(lv.bs_slot + set) != LH_NOSLOT;
}

__device__ __forceinline__ void last_pair(const JQuery &q, const JDepth &D, const uint32_t *posF, uint32_t capF,
                                          uint32_t i, LastPair &P) {
    uint32_t lo0, hi0, set0, lo1, hi1, set1;
    bool bs0, bs1;
    pair_side(q, D, posF, capF, i, 0, lo0, hi0, set0, bs0);
    pair_side(q, D, posF, capF, i, 1, lo1, hi1, set1, bs1);
    const bool swap = hi1 - lo1 < hi0 - lo0;
    P.pS = swap ? 1u : 0u;
    P.pT = swap ? 0u : 1u;
    P.sLo = swap ? lo1 : lo0; P.sHi = swap ? hi1 : hi0; P.sSet = swap ? set1 : set0;
    P.tLo = swap ? lo0 : lo1; P.tHi = swap ? hi0 : hi1; P.tSet = swap ? set0 : set1;
    const bool bsS = swap ? bs1 : bs0, bsT = swap ? bs0 : bs1;
    const uint64_t sn = P.sHi - P.sLo, tn = P.tHi - P.tLo;
    const bool close = tn <= (uint64_t)kMergeRatio * sn;
    if (bsT) P.kind = K_SCAN_S;
    else if (!bsS) P.kind = close ? K_MERGE : K_SCAN_S;
    else P.kind = close ? K_SCAN_T : K_SCAN_S;
    P.work = P.kind == K_MERGE ? sn + tn : P.kind == K_SCAN_S ? sn : tn;
    P.nseg = (P.work + kSegWork - 1) / kSegWork;
}

// Merge-path split: the number of A elements among the first `diag`
// elements of the merge of sorted A (s) and B (t), A first on equal values.
__device__ __forceinline__ uint32_t merge_split(const uint32_t *A, uint32_t s, const uint32_t *B, uint32_t t,
                                                uint64_t diag) {
    uint32_t lo = diag > t ? (uint32_t)(diag - t) : 0u;
    uint32_t hi = (uint32_t)(diag < s ? diag : (uint64_t)s);
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(A + mid) <= __ldg(B + (diag - mid - 1))) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// |A[a0, a1) ∩ B[b0, b1)| by one warp (all lanes, uniform bounds).  Every
// round loads a window of up to 32 elements of each; m, the smaller of the
// windows' last elements, bounds what this round settles: an A element <= m
// has its match, if any, inside B's window, and B elements <= m can match no
// later A element.  At least one window is used up per round.
__device__ __forceinline__ uint32_t warp_merge_count(const uint32_t *A, uint32_t a0, uint32_t a1, const uint32_t *B,
                                                     uint32_t b0, uint32_t b1, uint32_t lane) {
    uint32_t cnt = 0;
    while (a0 < a1 && b0 < b1) {
        const uint32_t na = min(32u, a1 - a0), nb = min(32u, b1 - b0);
        const bool va = lane < na, vb = lane < nb;
        const uint32_t a = va ? __ldg(A + a0 + lane) : 0xFFFFFFFFu;
        const uint32_t b = vb ? __ldg(B + b0 + lane) : 0xFFFFFFFFu;
        const uint32_t m = min(__shfl_sync(LH_FULL, a, na - 1), __shfl_sync(LH_FULL, b, nb - 1));
        // lower bound of a among B's window (lanes past nb hold the maximum)
        uint32_t pos = 0;
#pragma unroll
        for (uint32_t st = 16; st > 0; st >>= 1)
            if (__shfl_sync(LH_FULL, b, pos + st - 1) < a) pos += st;
        // every lane takes part in the shuffle (pos < 32 always); only then
        // is the result filtered
        const uint32_t bp = __shfl_sync(LH_FULL, b, pos);
        const bool hit = va && pos < nb && bp == a && a <= m;
        cnt += __popc(__ballot_sync(LH_FULL, hit));
        a0 += __popc(__ballot_sync(LH_FULL, va && a <= m));
        b0 += __popc(__ballot_sync(LH_FULL, vb && b <= m));
    }
    return cnt;
}

// nF_dev, when given, holds the frontier's real size (the previous depth's
// survivor counter, never read back to the host); entries from there up to
// nF are padding and get size 0.
__global__ void k_sizes(JQuery q, uint32_t d, const uint32_t *posF, uint32_t nF, const uint32_t *nF_dev,
                        uint32_t capF, uint32_t *size, uint8_t *drv, unsigned long long *elems, uint64_t *items,
                        unsigned long long *n_items, uint64_t cap_items) {
    const JDepth &D = q.D[d];
    const uint32_t n_real = nF_dev ? min(__ldg(nF_dev), nF) : nF;
    uint64_t local = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += gridDim.x * blockDim.x) {
        if (i >= n_real) {
            size[i] = 0;
            drv[i] = 0;
            continue;
        }
        uint32_t best = 0xFFFFFFFFu, bi = 0xFF;
        uint32_t flat_n = 0xFFFFFFFFu, flat_p = 0xFF;
        for (uint32_t p = 0; p < D.np; ++p) {
            const JEdge &E = q.E[D.e[p]];
            if (E.is_flat) {
                if (E.flat_n < flat_n) { flat_n = E.flat_n; flat_p = p; }
                continue;
            }
            uint32_t L = D.lvl[p];
            uint32_t parent = L ? posF[(uint64_t)D.e[p] * capF + i] : 0u;
            uint32_t lo, hi;
            lh_set_range(E.t, L, parent, lo, hi);
            uint32_t sz = hi - lo;
            local += sz;
            if (sz < best) { best = sz; bi = p; }
        }
        if (bi == 0xFF) { best = flat_n; bi = flat_p; }
        if (items != nullptr && best >= kWarpMinSet) {
            // a large pair of sets at the last COUNT attribute: its work
            // items go to k_count_pairs, and it drives no candidates here.
            // When the item list is full the entry stays on this path (the
            // slots it reserved below the capacity are marked empty).
            LastPair P;
            last_pair(q, D, posF, capF, i, P);
            const unsigned long long at = atomicAdd(n_items, (unsigned long long)P.nseg);
            if (at + P.nseg <= cap_items) {
                for (uint64_t g = 0; g < P.nseg; ++g) items[at + g] = ((uint64_t)i << 24) | g;
                best = 0;
            } else {
                for (uint64_t g = at; g < cap_items && g < at + P.nseg; ++g) items[g] = kNoItem;
            }
        }
        size[i] = best;
        drv[i] = (uint8_t)bi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(LH_FULL, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(elems, (unsigned long long)local);
}

// Work items of the large last-attribute pairs (see kWarpMinSet): one warp
// per item, grid-strided; item = entry << 24 | segment.
__global__ void __launch_bounds__(kThreads) k_count_pairs(JQuery q, uint32_t d, const uint32_t *posF, uint32_t capF,
                                                          const uint64_t *items, uint64_t n_items,
                                                          unsigned long long *count, unsigned long long *visited) {
    const JDepth &D = q.D[d];
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long cnt = 0, vis = 0;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_items; w += nw) {
        const uint64_t it = __ldg((const unsigned long long *)items + w);
        if (it == kNoItem) continue;
        const uint32_t i = (uint32_t)(it >> 24);
        const uint64_t g = it & 0xFFFFFFull;
        LastPair P;
        last_pair(q, D, posF, capF, i, P);
        const JEdge &ES = q.E[D.e[P.pS]];
        const JEdge &ET = q.E[D.e[P.pT]];
        const uint32_t LS = D.lvl[P.pS], LT = D.lvl[P.pT];
        const uint32_t *S = ES.t.lv[LS].vals + P.sLo;
        const uint32_t *T = ET.t.lv[LT].vals + P.tLo;
        const uint32_t sn = P.sHi - P.sLo, tn = P.tHi - P.tLo;
        const uint64_t w0 = g * kSegWork, w1 = (w0 + kSegWork < P.work) ? w0 + kSegWork : P.work;
        if (P.kind == K_MERGE) {
            const uint32_t ia0 = merge_split(S, sn, T, tn, w0), ia1 = merge_split(S, sn, T, tn, w1);
            const uint32_t ib0 = (uint32_t)(w0 - ia0), ib1 = (uint32_t)(w1 - ia1);
            // S elements of this item; a match of the last one may be T[ib1]
            const uint32_t bend = min(ib1 + 1, tn);
            cnt += warp_merge_count(S, ia0, ia1, T, ib0, bend, lane);
            vis += (ia1 - ia0) + (bend - ib0);
        } else {
            // lanes take the elements [w0, w1) of the scanned set X and probe
            // the other set Y
            const bool scan_s = P.kind == K_SCAN_S;
            const uint32_t *X = scan_s ? S : T;
            const JEdge &EY = scan_s ? ET : ES;
            const uint32_t LY = scan_s ? LT : LS;
            const uint32_t ylo = scan_s ? P.tLo : P.sLo, yhi = scan_s ? P.tHi : P.sHi;
            const uint32_t yset = scan_s ? P.tSet : P.sSet;
            const DLevel &ly = EY.t.lv[LY];
            const bool ybs = ly.bs_slot != nullptr && __ldg(ly.bs_slot + yset) != LH_NOSLOT;
            uint32_t lb = ylo;   // lower end of the uint search: the warp's previous elements are smaller
            for (uint64_t k = w0; k < w1; k += 32) {
                const uint32_t nv = (w1 - k < 32) ? (uint32_t)(w1 - k) : 32u;
                const bool v = lane < nv;
                const uint32_t x = v ? __ldg(X + k + lane) : 0u;
                bool hit = false;
                if (ybs) {
                    uint32_t pos;
                    hit = v && lh_probe(EY.t, LY, yset, ylo, yhi, x, &pos);
                } else {
                    const uint32_t p = v ? lh_lower_bound(ly.vals, lb, yhi, x) : yhi;
                    hit = v && p < yhi && __ldg(ly.vals + p) == x;
                    lb = __shfl_sync(LH_FULL, p, nv - 1);
                }
                cnt += __popc(__ballot_sync(LH_FULL, hit));
            }
            vis += 2 * (w1 - w0);
        }
    }
    if (lane == 0 && cnt) atomicAdd(count, cnt);
    if (lane == 0 && vis) atomicAdd(visited, vis);
}

// The root frontier entry (depth 0) as k_sizes and the scan would leave it.
__global__ void k_root(uint32_t *size, uint8_t *drv, uint64_t *off, uint32_t best, uint32_t bi,
                       unsigned long long el, unsigned long long *elems) {
    size[0] = best;
    drv[0] = (uint8_t)bi;
    off[0] = 0;
    off[1] = best;
    if (el) atomicAdd(elems, el);
}

struct ExpandOut {
    uint32_t *posO;
    uint32_t capO;
    uint32_t *gvO;
    uint32_t *counter;           // survivors emitted
    unsigned long long *count;   // COUNT without groups
    double *gsum;
    unsigned long long *gcount;
    uint32_t *status;            // context status word (out-of-domain GROUP BY values)
};

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_expand(JQuery q, uint32_t d, const uint32_t *posF,
                                                     const uint32_t *gvF, uint32_t nF, uint32_t capF,
                                                     const uint64_t *off, const uint8_t *drv,
                                                     uint64_t c0, uint64_t c1, ExpandOut o) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const JDepth &D = q.D[d];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const bool use_smem = MODE == M_AGG && q.gmode == G_DENSE && q.ngroups <= kSmemGroupsMax;
    const bool use_priv = MODE == M_AGG && q.gmode == G_PRIVATE;
    // dense:   float2 tab[nwarps][ngroups], uint32 tcnt[nwarps][ngroups], stage
    // private: u64 pkey[nwarps][P], float phi, plo [nwarps][P], uint32 pcnt[nwarps][P], stage
    float2 *tab = (float2 *)smem_raw;
    uint32_t *tcnt = (uint32_t *)(tab + (use_smem ? (size_t)nwarps * q.ngroups : 0));
    unsigned long long *pkey = (unsigned long long *)smem_raw;
    float *phi = (float *)(pkey + (use_priv ? (size_t)nwarps * kPrivSlots : 0));
    float *plo = phi + (use_priv ? (size_t)nwarps * kPrivSlots : 0);
    uint32_t *pcnt = (uint32_t *)(plo + (use_priv ? (size_t)nwarps * kPrivSlots : 0));
    float *stage_h = use_priv ? (float *)(pcnt + (size_t)nwarps * kPrivSlots)
                              : (float *)(tcnt + (use_smem ? (size_t)nwarps * q.ngroups : 0));
    float *stage_l = stage_h + nwarps * 32;
    if (use_smem) {
        for (uint32_t k = threadIdx.x; k < nwarps * q.ngroups; k += blockDim.x) {
            tab[k] = make_float2(0.f, 0.f);
            tcnt[k] = 0;
        }
        __syncthreads();
    }
    if (use_priv) {
        for (uint32_t k = threadIdx.x; k < nwarps * kPrivSlots; k += blockDim.x) {
            pkey[k] = kPrivEmpty;
            phi[k] = 0.f;
            plo[k] = 0.f;
            pcnt[k] = 0;
        }
        __syncthreads();
    }
    __shared__ uint64_t s_win[kWin];
    __shared__ uint32_t s_ent[2];
    uint32_t my_count = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = c0 + (uint64_t)blockIdx.x * blockDim.x; base < c1; base += stride) {
        const uint64_t c = base + threadIdx.x;
        bool ok = c < c1;
        uint32_t i = 0, x = 0;
        uint32_t npos[LH_MAX_EDGES];
        __syncthreads();   // the previous iteration is done with the window
        if (threadIdx.x == 0) {
            const uint32_t e0 = find_entry(off, nF, base);
            s_ent[0] = e0;
            s_ent[1] = find_entry(off, nF, min(base + blockDim.x, c1) - 1, e0);
        }
        __syncthreads();
        const uint32_t e0 = s_ent[0], win = s_ent[1] - e0 + 1;
        if (win <= kWin) {
            for (uint32_t t = threadIdx.x; t < win; t += blockDim.x) s_win[t] = __ldg(off + e0 + t);
            __syncthreads();
        }
        if (ok) {
            if (win <= kWin) {
                uint32_t lo = 0, hi = win;  // s_win[lo] <= c < s_win[hi] (hi = win: beyond the window)
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s_win[mid] <= c) lo = mid;
                    else hi = mid;
                }
                i = e0 + lo;
            } else {
                i = find_entry(off, e0 + win, c, e0);
            }
            const uint32_t j = (uint32_t)(c - off[i]);
            const uint32_t p0 = drv[i];
            const JEdge &E0 = q.E[D.e[p0]];
            if (E0.is_flat) {
                x = j;
                npos[p0] = j;
            } else {
                const uint32_t L0 = D.lvl[p0];
                const uint32_t parent = L0 ? posF[(uint64_t)D.e[p0] * capF + i] : 0u;
                uint32_t lo, hi;
                lh_set_range(E0.t, L0, parent, lo, hi);
                x = __ldg(E0.t.lv[L0].vals + lo + j);
                npos[p0] = lo + j;
            }
            for (uint32_t p = 0; p < D.np && ok; ++p) {
                if (p == p0) continue;
                const JEdge &E = q.E[D.e[p]];
                if (E.is_flat) {
                    ok = x < E.flat_n;
                    npos[p] = x;
                    continue;
                }
                const uint32_t L = D.lvl[p];
                const uint32_t parent = L ? posF[(uint64_t)D.e[p] * capF + i] : 0u;
                uint32_t lo, hi;
                lh_set_range(E.t, L, parent, lo, hi);
                ok = lh_probe(E.t, L, L ? parent : 0u, lo, hi, x, &npos[p]);
            }
        }
        if (MODE == M_EMIT) {
            const uint32_t ball = __ballot_sync(LH_FULL, ok);
            uint32_t basep = 0;
            if (lane == 0 && ball) basep = atomicAdd(o.counter, (uint32_t)__popc(ball));
            basep = __shfl_sync(LH_FULL, basep, 0);
            if (ok) {
                const uint32_t slot = basep + __popc(ball & ((1u << lane) - 1u));
                for (uint32_t e = 0; e < q.ne; ++e) {
                    uint32_t v = 0;
                    bool part = false;
                    for (uint32_t p = 0; p < D.np; ++p)
                        if (D.e[p] == e) { v = npos[p]; part = true; }
                    if (!part) v = (d > 0) ? posF[(uint64_t)e * capF + i] : 0u;
                    o.posO[(uint64_t)e * o.capO + slot] = v;
                }
                for (uint32_t g = 0; g < q.ngc; ++g) {
                    if (!q.g_is_key[g]) continue;
                    const uint32_t s = q.g_slot[g];
                    uint32_t v = (q.g_depth[g] == d) ? x : ((d > 0) ? gvF[(uint64_t)s * capF + i] : 0u);
                    o.gvO[(uint64_t)s * o.capO + slot] = v;
                }
            }
        } else if (MODE == M_COUNT) {
            my_count += ok ? 1u : 0u;
        } else {
            // leaf positions of every relation, the group and the product term
            uint32_t g = 0;
            uint32_t kv[kMaxG];
            unsigned long long K = kPrivEmpty;
            float th = 1.f, tl = 0.f;
            if (ok) {
                uint32_t lp[LH_MAX_EDGES];
                for (uint32_t e = 0; e < q.ne; ++e) {
                    lp[e] = (d > 0) ? posF[(uint64_t)e * capF + i] : 0u;
                    for (uint32_t p = 0; p < D.np; ++p)
                        if (D.e[p] == e) lp[e] = npos[p];
                }
                bool in_domain = true;
                K = 0;
                for (uint32_t k = 0; k < q.ngc; ++k) {
                    uint32_t gv;
                    if (q.g_is_key[k])
                        gv = (q.g_depth[k] == d) ? x : gvF[(uint64_t)q.g_slot[k] * capF + i];
                    else
                        gv = (uint32_t)__ldg(q.g_col[k] + lp[q.g_edge[k]]);
                    // a value outside a declared [0, card) (a negative int32
                    // reads as a huge unsigned value) breaks the caller's
                    // contract: the tuple is left out and the error surfaces
                    // at the wait
                    const bool in = q.g_card[k] == 0 || gv < q.g_card[k];
                    in_domain = in_domain && in;
                    kv[k] = gv;
                    g = g * q.g_card[k] + (in ? gv : 0u);
                    K |= (unsigned long long)gv << q.g_shift[k];
                }
                if (!in_domain) {
                    lh_set_status(o.status, LH_EINVAL);
                    ok = false;
                }
                if (!q.count_only) {
                    for (uint32_t e = 0; e < q.ne; ++e) {
                        const JEdge &E = q.E[e];
                        if (E.anno_kind == 0) continue;
                        float ah = E.is_flat ? __ldg(E.flat + lp[e]) : __ldg(E.a_hi + lp[e]);
                        float al = (E.anno_kind == 2) ? __ldg(E.a_lo + lp[e]) : 0.f;
                        float ph, pe;
                        lh_two_prod(th, ah, ph, pe);
                        tl = pe + fmaf(th, al, tl * ah);
                        th = ph;
                    }
                }
            }
            if (use_priv) {
                // lanes with one key tuple merge their terms; the leader
                // upserts into this warp's table (claims by CAS, so two
                // leaders never share a slot), spilling to the shared table
                // when the warp's table is full
                const unsigned long long key = ok ? K : kPrivEmpty;
                const uint32_t peers = __match_any_sync(LH_FULL, key);
                stage_h[warp * 32 + lane] = th;
                stage_l[warp * 32 + lane] = tl;
                __syncwarp();
                if (ok && (peers & ((1u << lane) - 1u)) == 0) {
                    float sh = 0.f, sl = 0.f;
                    uint32_t m = peers;
                    while (m) {
                        const int s = __ffs(m) - 1;
                        m &= m - 1;
                        lh_pair_add(sh, sl, stage_h[warp * 32 + s], stage_l[warp * 32 + s]);
                    }
                    unsigned long long *wk = pkey + (size_t)warp * kPrivSlots;
                    uint32_t slot = (uint32_t)mix64(K) & (kPrivSlots - 1);
                    bool placed = false;
                    for (uint32_t probe = 0; probe < kPrivSlots; ++probe) {
                        const unsigned long long prev = atomicCAS(wk + slot, kPrivEmpty, K);
                        if (prev == kPrivEmpty || prev == K) {
                            const size_t c = (size_t)warp * kPrivSlots + slot;
                            float ch = phi[c], cl = plo[c];
                            lh_pair_add(ch, cl, sh, sl);
                            phi[c] = ch;
                            plo[c] = cl;
                            pcnt[c] += __popc(peers);
                            placed = true;
                            break;
                        }
                        slot = (slot + 1) & (kPrivSlots - 1);
                    }
                    if (!placed) ht_upsert(q.ht, q.ngc, kv, (double)sh + (double)sl, __popc(peers), o.status);
                }
                __syncwarp();
            } else if (MODE == M_AGG && q.gmode == G_SHARED) {
                if (ok) ht_upsert(q.ht, q.ngc, kv, (double)th + (double)tl, 1ull, o.status);
            } else if (use_smem) {
                const uint32_t key = ok ? g : 0xFFFFFFFFu;
                const uint32_t peers = __match_any_sync(LH_FULL, key);
                stage_h[warp * 32 + lane] = th;
                stage_l[warp * 32 + lane] = tl;
                __syncwarp();
                if (ok && (peers & ((1u << lane) - 1u)) == 0) {  // leader of its group
                    float sh = 0.f, sl = 0.f;
                    uint32_t m = peers;
                    while (m) {
                        const int s = __ffs(m) - 1;
                        m &= m - 1;
                        lh_pair_add(sh, sl, stage_h[warp * 32 + s], stage_l[warp * 32 + s]);
                    }
                    float2 &cell = tab[(size_t)warp * q.ngroups + g];
                    float ch = cell.x, cl = cell.y;
                    lh_pair_add(ch, cl, sh, sl);
                    cell = make_float2(ch, cl);
                    tcnt[(size_t)warp * q.ngroups + g] += __popc(peers);
                }
                __syncwarp();
            } else if (ok) {
                atomicAdd(o.gsum + g, (double)th + (double)tl);
                atomicAdd(o.gcount + g, 1ull);
            }
        }
    }
    if (MODE == M_COUNT) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) my_count += __shfl_xor_sync(LH_FULL, my_count, s);
        if (lane == 0 && my_count) atomicAdd(o.count, (unsigned long long)my_count);
    }
    if (use_priv) {
        // every warp merges its own table into the shared one
        __syncwarp();
        for (uint32_t sl = lane; sl < kPrivSlots; sl += 32) {
            const size_t c = (size_t)warp * kPrivSlots + sl;
            if (pkey[c] == kPrivEmpty) continue;
            uint32_t kv[kMaxG];
            unpack_key(q, pkey[c], kv);
            ht_upsert(q.ht, q.ngc, kv, (double)phi[c] + (double)plo[c], pcnt[c], o.status);
        }
    }
    if (use_smem) {
        __syncthreads();
        for (uint32_t g = threadIdx.x; g < q.ngroups; g += blockDim.x) {
            float sh = 0.f, sl = 0.f;
            uint32_t cn = 0;
            for (uint32_t w = 0; w < nwarps; ++w) {
                float2 cell = tab[(size_t)w * q.ngroups + g];
                lh_pair_add(sh, sl, cell.x, cell.y);
                cn += tcnt[(size_t)w * q.ngroups + g];
            }
            if (cn) {
                atomicAdd(o.gsum + g, (double)sh + (double)sl);
                atomicAdd(o.gcount + g, (unsigned long long)cn);
            }
        }
    }
}

struct Driver {
    lh_ctx *ctx;
    JQuery q;
    lh_result *r;
    uint32_t cap;
    uint32_t n_keygroups;
    uint32_t mode_last;   // M_COUNT or M_AGG
    bool shortcut_last;   // last depth has one set and nothing to aggregate: add sizes
    bool pairs_last;      // last depth counts two trie sets: large pairs go to k_count_pairs
    unsigned grid_pairs;
    size_t smem_bytes;
    unsigned grid_expand;
    std::chrono::steady_clock::time_point t0;
    double deadline_ms;

    lh_status check_time() {
        if (deadline_ms <= 0) return LH_OK;
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > deadline_ms) return lh_fail(ctx, LH_ETIMEOUT, "join exceeded its %.1f ms budget", deadline_ms);
        return LH_OK;
    }

    // nF: the frontier's size, or an upper bound when nF_dev (a device
    // counter holding the real size) is given
    lh_status run(uint32_t d, const uint32_t *posF, const uint32_t *gvF, uint32_t nF, uint32_t capF,
                  const uint32_t *nF_dev = nullptr) {
        if (nF == 0) return LH_OK;
        LH_TRY(check_time());
        uint32_t *size = nullptr;
        uint8_t *drvb = nullptr;
        uint64_t *off = nullptr;
        const bool last = d + 1 == q.nd;
        const bool pairs = last && pairs_last;
        uint64_t *items = nullptr;
        const uint64_t cap_items = pairs ? (uint64_t)nF + (1u << 18) : 0;
        // off[nF]: the candidate total; off[nF + 1]: the pair work items
        lh_status s = lh_alloc(ctx, &size, nF);
        if (s == LH_OK) s = lh_alloc(ctx, &drvb, nF);
        if (s == LH_OK) s = lh_alloc(ctx, &off, (size_t)nF + 2);
        if (s == LH_OK && pairs) s = lh_alloc(ctx, &items, cap_items);
        uint64_t rb[2] = {0, 0};
        if (s == LH_OK) {
            if (pairs && cudaMemsetAsync(off + nF + 1, 0, sizeof(uint64_t), ctx->stream) != cudaSuccess)
                s = lh_fail(ctx, LH_ECUDA, "memset failed");
        }
        const bool root = d == 0 && posF == nullptr && !last;
        if (s == LH_OK && root) {
            // the root's sets are the level-0 sets, whose sizes the host
            // knows: the driver is picked here, with no sizes kernel, scan
            // or readback
            const JDepth &D = q.D[0];
            uint32_t best = 0xFFFFFFFFu, bi = 0xFF, flat_n = 0xFFFFFFFFu, flat_p = 0xFF;
            unsigned long long el = 0;
            for (uint32_t p = 0; p < D.np; ++p) {
                const JEdge &E = q.E[D.e[p]];
                if (E.is_flat) {
                    if (E.flat_n < flat_n) { flat_n = E.flat_n; flat_p = p; }
                    continue;
                }
                const uint32_t sz = E.t.lv[0].n;
                el += sz;
                if (sz < best) { best = sz; bi = p; }
            }
            if (bi == 0xFF) { best = flat_n; bi = flat_p; }
            LH_TRACED(ctx, "k_root", k_root<<<1, 1, 0, ctx->stream>>>(size, drvb, off, best, bi, el,
                                                                       (unsigned long long *)r->d_elems));
            rb[0] = best;
        } else if (s == LH_OK) {
            unsigned g = (unsigned)std::min<uint64_t>(lh_blocks(nF, kThreads), (uint64_t)ctx->num_sms * 8);
            LH_TRACED(ctx, "k_sizes", k_sizes<<<g, kThreads, 0, ctx->stream>>>(q, d, posF, nF, nF_dev, capF, size, drvb,
                                                     (unsigned long long *)r->d_elems, items,
                                                     (unsigned long long *)(off + nF + 1), cap_items));
            s = lh_scan_u32_to_u64(ctx, size, off, nF);
            if (s == LH_OK) s = lh_readback(ctx, off + nF, (pairs ? 2 : 1) * sizeof(uint64_t), rb);
        }
        const uint64_t total = rb[0], n_items = std::min<uint64_t>(rb[1], cap_items);
        if (s == LH_OK && !(last && shortcut_last)) r->visited += total * q.D[d].np;
        if (s == LH_OK && last) {
            if (n_items) {
                const unsigned g = (unsigned)std::min<uint64_t>(lh_blocks(n_items * 32, kThreads), grid_pairs);
                LH_TRACED(ctx, "k_count_pairs", k_count_pairs<<<g, kThreads, 0, ctx->stream>>>(
                                                    q, d, posF, capF, items, n_items, (unsigned long long *)r->d_count,
                                                    (unsigned long long *)r->d_elems + 1));
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "count pairs: %s", cudaGetErrorString(e));
            }
            if (s != LH_OK) {
            } else if (shortcut_last) {
                r->host_count += total;
            } else if (total) {
                ExpandOut o = {};
                o.count = (unsigned long long *)r->d_count;
                o.gsum = r->d_gsum;
                o.gcount = (unsigned long long *)r->d_gcount;
                o.status = ctx->d_status;
                // the last attribute's candidates in launches of at most
                // kLastChunk, so that a time budget can stop a join whose
                // frontier fans out into billions of candidates
                for (uint64_t c0 = 0; c0 < total && s == LH_OK; c0 += kLastChunk) {
                    if (c0) s = check_time();
                    if (s != LH_OK) break;
                    const uint64_t c1 = std::min<uint64_t>(total, c0 + kLastChunk);
                    if (mode_last == M_COUNT)
                        LH_TRACED(ctx, "k_expand", k_expand<M_COUNT><<<grid_expand, kThreads, 0, ctx->stream>>>(q, d, posF, gvF, nF, capF, off, drvb, c0, c1, o));
                    else
                        LH_TRACED(ctx, "k_expand", k_expand<M_AGG><<<grid_expand, kThreads, smem_bytes, ctx->stream>>>(q, d, posF, gvF, nF, capF, off, drvb, c0, c1, o));
                    cudaError_t e = cudaGetLastError();
                    if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "expand: %s", cudaGetErrorString(e));
                    if (s == LH_OK && deadline_ms > 0 && c1 < total) {
                        // the host clock only sees the time once the work is done
                        cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
                        if (e2 != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "expand: %s", cudaGetErrorString(e2));
                    }
                }
            }
        } else if (s == LH_OK) {
            for (uint64_t c0 = 0; c0 < total && s == LH_OK; c0 += cap) {
                const uint64_t c1 = std::min<uint64_t>(total, c0 + cap);
                const uint32_t capO = (uint32_t)(c1 - c0);
                uint32_t *posO = nullptr, *gvO = nullptr, *counter = nullptr;
                s = lh_alloc(ctx, &posO, (size_t)q.ne * capO);
                if (s == LH_OK) s = lh_alloc(ctx, &gvO, (size_t)std::max(1u, n_keygroups) * capO);
                if (s == LH_OK) s = lh_alloc(ctx, &counter, 1);
                uint32_t nO = 0;
                if (s == LH_OK) {
                    cudaMemsetAsync(counter, 0, sizeof(uint32_t), ctx->stream);
                    ExpandOut o = {};
                    o.posO = posO;
                    o.capO = capO;
                    o.gvO = gvO;
                    o.counter = counter;
                    unsigned g = (unsigned)std::min<uint64_t>(lh_blocks(c1 - c0, kThreads), grid_expand);
                    LH_TRACED(ctx, "k_expand", k_expand<M_EMIT><<<g, kThreads, 0, ctx->stream>>>(q, d, posF, gvF, nF, capF, off, drvb, c0, c1, o));
                    cudaError_t e = cudaGetLastError();
                    if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "expand: %s", cudaGetErrorString(e));
                }
                // a small chunk's survivors are not read back: the next depth
                // runs over the chunk's capacity and reads the real count on
                // the device (one host round trip fewer per depth)
                if (s == LH_OK && capO <= kPadFrontierMax) {
                    s = run(d + 1, posO, gvO, capO, capO, counter);
                } else {
                    if (s == LH_OK) s = lh_readback(ctx, counter, sizeof(uint32_t), &nO);
                    if (s == LH_OK) s = run(d + 1, posO, gvO, nO, capO);
                }
                lh_free(ctx, posO);
                lh_free(ctx, gvO);
                lh_free(ctx, counter);
            }
        }
        lh_free(ctx, size);
        lh_free(ctx, drvb);
        lh_free(ctx, off);
        lh_free(ctx, items);
        return s;
    }
};

}  // namespace

bool lh_key_order_for(const lh_query *q, const uint32_t *order, uint32_t n_attrs, uint32_t e,
                      uint32_t *key_order) {
    if (e >= q->n_edges) return false;
    const lh_edge &E = q->edges[e];
    uint32_t pos[LH_MAX_ATTRS];
    for (uint32_t a = 0; a < LH_MAX_ATTRS; ++a) pos[a] = 0xFFFFFFFFu;
    for (uint32_t k = 0; k < n_attrs; ++k) {
        if (order[k] >= LH_MAX_ATTRS) return false;
        pos[order[k]] = k;
    }
    uint32_t idx[LH_MAX_LEVELS];
    for (uint32_t c = 0; c < E.nattrs; ++c) {
        if (E.attrs[c] >= LH_MAX_ATTRS || pos[E.attrs[c]] == 0xFFFFFFFFu) return false;
        idx[c] = c;
    }
    std::sort(idx, idx + E.nattrs, [&](uint32_t x, uint32_t y) { return pos[E.attrs[x]] < pos[E.attrs[y]]; });
    for (uint32_t c = 0; c < E.nattrs; ++c) key_order[c] = idx[c];
    return true;
}

extern "C" lh_status lh_edge_key_order(const lh_query *q, const lh_plan_t *plan, uint32_t e,
                                       uint32_t *key_order) {
    if (!q || !plan || !key_order) return LH_EINVAL;
    return lh_key_order_for(q, plan->order, plan->n_attrs, e, key_order) ? LH_OK : LH_EINVAL;
}

lh_status lh_run_generic(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan,
                         lh_trie *const *tries, lh_result *r, double deadline_ms) {
    Driver dr;
    dr.ctx = ctx;
    dr.r = r;
    dr.t0 = std::chrono::steady_clock::now();
    dr.deadline_ms = deadline_ms;
    JQuery &jq = dr.q;
    memset(&jq, 0, sizeof(jq));
    jq.ne = q->n_edges;
    jq.nd = plan->n_attrs;
    // edges
    uint32_t edge_level_attr[LH_MAX_EDGES][LH_MAX_LEVELS];
    for (uint32_t e = 0; e < q->n_edges; ++e) {
        const lh_edge &E = q->edges[e];
        JEdge &J = jq.E[e];
        if (E.trie_slot < 0) {
            if (E.nattrs != 1 || !E.flat) return lh_fail(ctx, LH_EINVAL, "flat edge %u needs one attribute and a buffer", e);
            if (E.flat_n >= (1ull << 32)) return lh_fail(ctx, LH_EOVERFLOW, "flat edge too long");
            J.is_flat = 1;
            J.flat = E.flat;
            J.flat_n = (uint32_t)E.flat_n;
            J.anno_kind = (E.anno >= 0) ? 1 : 0;
            edge_level_attr[e][0] = E.attrs[0];
            continue;
        }
        const lh_trie *t = tries[E.trie_slot];
        if (!t) return lh_fail(ctx, LH_EINVAL, "edge %u: null trie", e);
        if (t->nlevels != E.nattrs) return lh_fail(ctx, LH_EINVAL, "edge %u: trie has %u levels, edge %u attributes", e, t->nlevels, E.nattrs);
        uint32_t want[LH_MAX_LEVELS];
        if (!lh_key_order_for(q, plan->order, plan->n_attrs, e, want)) return lh_fail(ctx, LH_EINVAL, "edge %u: attribute missing from plan", e);
        for (uint32_t l = 0; l < E.nattrs; ++l)
            if (t->key_order[l] != want[l]) return lh_fail(ctx, LH_EINVAL, "edge %u: trie key order does not follow the plan's attribute order", e);
        for (uint32_t l = 0; l < E.nattrs; ++l) {
            edge_level_attr[e][l] = E.attrs[t->key_order[l]];
            if (t->lv[l].n >= (1ull << 32) - 1) return lh_fail(ctx, LH_EOVERFLOW, "level too large");
        }
        J.t = lh_trie_dview(t);
        if (E.anno >= 0) {
            if ((uint32_t)E.anno >= t->nannos) return lh_fail(ctx, LH_EINVAL, "edge %u: no annotation column %d", e, E.anno);
            uint32_t ty = t->anno_type[E.anno];
            if (ty != LH_T_F32) return lh_fail(ctx, LH_EUNSUPPORTED, "edge %u: multiplied annotations must be f32", e);
            J.a_hi = (const float *)t->anno[E.anno];
            J.anno_kind = 1;
            // a price/discount trie stores the expression as (high, low) f32 columns 0 and 1
            if (E.anno == 0 && t->nannos == 2 && t->anno_type[1] == LH_T_F32) {
                J.a_lo = (const float *)t->anno[1];
                J.anno_kind = 2;
            }
        }
    }
    // depths
    for (uint32_t d = 0; d < plan->n_attrs; ++d) {
        JDepth &D = jq.D[d];
        const uint32_t v = plan->order[d];
        for (uint32_t e = 0; e < q->n_edges; ++e) {
            const uint32_t nl = q->edges[e].nattrs;
            for (uint32_t l = 0; l < nl; ++l)
                if (edge_level_attr[e][l] == v) {
                    D.e[D.np] = (uint8_t)e;
                    D.lvl[D.np] = (uint8_t)l;
                    D.np++;
                }
        }
        if (D.np == 0) return lh_fail(ctx, LH_EINVAL, "attribute %u is in no relation", v);
        // a relation's level must be bound right after its previous level's attribute
        for (uint32_t p = 0; p < D.np; ++p) {
            uint32_t e = D.e[p], l = D.lvl[p];
            if (l > 0) {
                uint32_t prev = edge_level_attr[e][l - 1];
                bool earlier = false;
                for (uint32_t k = 0; k < d; ++k) earlier |= plan->order[k] == prev;
                if (!earlier) return lh_fail(ctx, LH_EINVAL, "edge %u level order breaks the plan", e);
            }
        }
    }
    // groups
    jq.ngc = q->n_group;
    jq.ngroups = 1;
    dr.n_keygroups = 0;
    if (q->n_group > kMaxG) return lh_fail(ctx, LH_EUNSUPPORTED, "at most %d GROUP BY columns", kMaxG);
    bool all_cards = true;
    uint64_t dense_groups = 1;
    uint32_t packed_bits = 0;
    uint64_t group_space = 1;  // bound on the distinct key tuples (sizes the shared table)
    for (uint32_t k = 0; k < q->n_group; ++k) {
        const lh_group &G = q->group[k];
        jq.g_card[k] = G.card;
        all_cards = all_cards && G.card > 0;
        dense_groups = std::min<uint64_t>(dense_groups * std::max<uint32_t>(G.card, 1u), 1ull << 40);
        jq.g_shift[k] = packed_bits;
        uint32_t bits = 32;
        if (G.card > 0) {
            bits = 1;
            while (bits < 32 && (1ull << bits) < G.card) ++bits;
        }
        packed_bits += bits;
        if (G.anno < 0) {
            jq.g_is_key[k] = 1;
            jq.g_slot[k] = dr.n_keygroups++;
            bool found = false;
            for (uint32_t d = 0; d < plan->n_attrs; ++d)
                if (plan->order[d] == G.attr) { jq.g_depth[k] = d; found = true; }
            if (!found) return lh_fail(ctx, LH_EINVAL, "group %u: attribute not in plan", k);
            // distinct values of a key attribute: at most the smallest level
            // holding it among the relations that contain it
            uint64_t dom = UINT64_MAX;
            for (uint32_t e = 0; e < q->n_edges; ++e) {
                const lh_edge &E = q->edges[e];
                if (E.trie_slot < 0) continue;
                const lh_trie *t = tries[E.trie_slot];
                for (uint32_t l = 0; l < t->nlevels; ++l)
                    if (E.attrs[t->key_order[l]] == G.attr) dom = std::min<uint64_t>(dom, t->lv[l].n);
            }
            if (G.card > 0) dom = std::min<uint64_t>(dom, G.card);
            group_space = std::min<uint64_t>(group_space * std::max<uint64_t>(1, dom == UINT64_MAX ? 1 : dom), 1ull << 40);
        } else {
            if (G.edge >= q->n_edges || q->edges[G.edge].trie_slot < 0) return lh_fail(ctx, LH_EINVAL, "group %u: bad edge", k);
            const lh_trie *t = tries[q->edges[G.edge].trie_slot];
            if ((uint32_t)G.anno >= t->nannos || (t->anno_type[G.anno] != LH_T_I32 && t->anno_type[G.anno] != LH_T_U32))
                return lh_fail(ctx, LH_EINVAL, "group %u: needs an int32 annotation column", k);
            jq.g_edge[k] = G.edge;
            jq.g_col[k] = (const int32_t *)t->anno[G.anno];
            // distinct values of an annotation column: at most its card, at
            // most the rows of its relation
            const uint64_t dom = G.card > 0 ? std::min<uint64_t>(G.card, t->lv[t->nlevels - 1].n) : t->lv[t->nlevels - 1].n;
            group_space = std::min<uint64_t>(group_space * std::max<uint64_t>(1, dom), 1ull << 40);
        }
    }
    // implementation (Section 5): dense arrays for small declared domains,
    // else private tables for key tuples of at most three values, the shared
    // table for wider ones
    uint32_t impl = q->group_impl;
    const bool dense_ok = all_cards && q->n_group <= 2 && dense_groups <= (1ull << 26);
    if (impl == LH_GROUP_AUTO)
        impl = q->n_group == 0 || dense_ok ? LH_GROUP_DENSE : (q->n_group <= 3 && packed_bits <= 63) ? LH_GROUP_PRIVATE
                                                                                                     : LH_GROUP_SHARED;
    if (q->n_group == 0) impl = LH_GROUP_DENSE;
    if (impl == LH_GROUP_DENSE && !dense_ok)
        return lh_fail(ctx, LH_EUNSUPPORTED, "dense GROUP BY needs at most two columns with declared cards and a domain <= 2^26");
    if (impl == LH_GROUP_PRIVATE && packed_bits > 63)
        return lh_fail(ctx, LH_EUNSUPPORTED, "private GROUP BY tables need the packed key (%u bits) to fit 63 bits", packed_bits);
    if (impl > LH_GROUP_SHARED) return lh_fail(ctx, LH_EINVAL, "unknown group_impl %u", impl);
    jq.gmode = impl == LH_GROUP_DENSE ? G_DENSE : impl == LH_GROUP_PRIVATE ? G_PRIVATE : G_SHARED;
    if (jq.gmode == G_DENSE) jq.ngroups = (uint32_t)dense_groups;
    r->group_impl = impl;
    const bool is_count = q->semiring == LH_COUNT_U64;
    jq.count_only = is_count ? 1 : 0;
    const JDepth &DL = jq.D[jq.nd - 1];
    uint32_t nonflat = 0;
    for (uint32_t p = 0; p < DL.np; ++p) nonflat += jq.E[DL.e[p]].is_flat ? 0 : 1;
    dr.mode_last = (is_count && q->n_group == 0) ? M_COUNT : M_AGG;
    dr.shortcut_last = dr.mode_last == M_COUNT && DL.np == 1 && nonflat == 1;
    if (q->isect_impl > LH_ISECT_PROBE) return lh_fail(ctx, LH_EINVAL, "unknown isect_impl %u", q->isect_impl);
    dr.pairs_last = dr.mode_last == M_COUNT && DL.np == 2 && nonflat == 2 && q->isect_impl == LH_ISECT_AUTO;
    {
        int pp = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pp, k_count_pairs, kThreads, 0);
        dr.grid_pairs = (unsigned)(ctx->num_sms * std::max(1, pp));
    }
    dr.cap = 1u << 22;
    dr.smem_bytes = 0;
    int per_sm = 4;
    const size_t stage = (size_t)(kThreads / 32) * 32 * 2 * sizeof(float);
    if (dr.mode_last == M_AGG && jq.gmode == G_DENSE && jq.ngroups <= kSmemGroupsMax)
        dr.smem_bytes = (size_t)(kThreads / 32) * jq.ngroups * (sizeof(float2) + sizeof(uint32_t)) + stage;
    else if (dr.mode_last == M_AGG && jq.gmode == G_PRIVATE)
        dr.smem_bytes = (size_t)(kThreads / 32) * kPrivSlots * (8 + 4 + 4 + 4) + stage;
    if (dr.smem_bytes) {
        cudaFuncSetAttribute(k_expand<M_AGG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dr.smem_bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand<M_AGG>, kThreads, dr.smem_bytes);
        if (per_sm < 1) per_sm = 1;
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand<M_COUNT>, kThreads, 0);
        if (per_sm < 1) per_sm = 1;
    }
    dr.grid_expand = (unsigned)(ctx->num_sms * per_sm);
    // results
    r->ngroups = (dr.mode_last == M_AGG && jq.gmode == G_DENSE) ? jq.ngroups : 0;
    // count, elements, elements read by k_count_pairs: one block, read back at once
    LH_TRY(res_alloc(ctx, r, &r->d_count, 3));
    r->d_elems = r->d_count + 1;
    LH_CU(cudaMemsetAsync(r->d_count, 0, 3 * sizeof(uint64_t), ctx->stream));
    if (r->ngroups) {
        LH_TRY(res_alloc(ctx, r, &r->d_gsum, r->ngroups));
        LH_TRY(res_alloc(ctx, r, &r->d_gcount, r->ngroups));
        LH_CU(cudaMemsetAsync(r->d_gsum, 0, r->ngroups * sizeof(double), ctx->stream));
        LH_CU(cudaMemsetAsync(r->d_gcount, 0, r->ngroups * sizeof(uint64_t), ctx->stream));
    }
    if (dr.mode_last == M_AGG && jq.gmode != G_DENSE) {
        // the shared table: twice the bound on distinct key tuples (the
        // product of the columns' domains: declared cards, else the distinct
        // values their relations can hold), clamped to [2^12, 2^24] slots,
        // unless the query gives a capacity
        uint64_t cap = q->group_capacity;
        if (cap == 0) cap = std::min<uint64_t>(std::max<uint64_t>(2 * group_space, 1ull << 12), 1ull << 24);
        uint64_t c2 = 1;
        while (c2 < cap) c2 <<= 1;
        if (c2 > (1ull << 31)) return lh_fail(ctx, LH_EUNSUPPORTED, "group_capacity above 2^31");
        HTab &H = jq.ht;
        H.cap = (uint32_t)c2;
        LH_TRY(res_alloc(ctx, r, &H.tag, c2));
        LH_TRY(res_alloc(ctx, r, &H.keys, c2 * std::max<uint32_t>(1u, q->n_group)));
        LH_TRY(res_alloc(ctx, r, &H.sum, c2));
        LH_TRY(res_alloc(ctx, r, &H.cnt, c2));
        LH_CU(cudaMemsetAsync(H.tag, 0, c2 * sizeof(unsigned long long), ctx->stream));
        LH_CU(cudaMemsetAsync(H.sum, 0, c2 * sizeof(double), ctx->stream));
        LH_CU(cudaMemsetAsync(H.cnt, 0, c2 * sizeof(unsigned long long), ctx->stream));
        r->ht_tag = H.tag;
        r->ht_keys = H.keys;
        r->ht_sum = H.sum;
        r->ht_cnt = H.cnt;
        r->ht_cap = H.cap;
        r->n_group_cols = q->n_group;
        r->hash_pending = true;
    }
    // depth 0 starts from the single empty prefix
    return dr.run(0, nullptr, nullptr, 1, 1);
}

// ------------------------------------------------------------------- C ABI

static bool is_spmv(const lh_query *q, const lh_plan_t *p) {
    if (q->n_edges != 2 || q->n_group != 1 || q->group[0].anno >= 0 || p->n_attrs != 2) return false;
    const lh_edge *A = nullptr, *X = nullptr;
    for (uint32_t e = 0; e < 2; ++e) (q->edges[e].trie_slot < 0 ? X : A) = &q->edges[e];
    if (!A || !X || A->nattrs != 2 || X->nattrs != 1 || A->anno != 0) return false;
    const uint32_t i = q->group[0].attr;
    return p->order[0] == i && p->order[1] == X->attrs[0] && A->attrs[0] == i && A->attrs[1] == X->attrs[0];
}

static bool is_spgemm(const lh_query *q, const lh_plan_t *p) {
    if (q->n_edges != 2 || q->n_group != 2 || p->n_attrs != 3) return false;
    if (q->group[0].anno >= 0 || q->group[1].anno >= 0) return false;
    const lh_edge &A = q->edges[0], &B = q->edges[1];
    if (A.trie_slot < 0 || B.trie_slot < 0 || A.nattrs != 2 || B.nattrs != 2 || A.anno != 0 || B.anno != 0) return false;
    const uint32_t i = A.attrs[0], j = A.attrs[1], k = B.attrs[1];
    return B.attrs[0] == j && q->group[0].attr == i && q->group[1].attr == k && p->order[0] == i &&
           p->order[1] == j && p->order[2] == k;
}

lh_status lh_join_dispatch(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan, lh_trie *const *tries,
                           lh_result **out, double deadline_ms) {
    if (!ctx || !q || !plan || !out) return lh_fail(ctx, LH_EINVAL, "null argument");
    *out = nullptr;
    if (q->n_edges == 0 || q->n_edges > LH_MAX_EDGES || plan->n_attrs == 0 || plan->n_attrs > LH_MAX_ATTRS ||
        plan->n_attrs != q->n_attrs)
        return lh_fail(ctx, LH_EINVAL, "bad query or plan sizes");
    for (uint32_t e = 0; e < q->n_edges; ++e)
        if (q->edges[e].nattrs == 0 || q->edges[e].nattrs > LH_MAX_LEVELS) return lh_fail(ctx, LH_EINVAL, "edge %u: bad arity", e);
    lh_result *r = new lh_result();
    r->semiring = q->semiring;
    lh_status s;
    uint32_t exec = q->exec;
    if (exec == LH_EXEC_AUTO) exec = is_spmv(q, plan) ? LH_EXEC_SPMV : is_spgemm(q, plan) ? LH_EXEC_SPGEMM : LH_EXEC_GENERIC;
    r->exec = exec;
    if (exec == LH_EXEC_SPMV) {
        if (!is_spmv(q, plan)) s = lh_fail(ctx, LH_EINVAL, "query is not an SpMV join-aggregate under this plan");
        else {
            const lh_edge *A = nullptr, *X = nullptr;
            for (uint32_t e = 0; e < 2; ++e) (q->edges[e].trie_slot < 0 ? X : A) = &q->edges[e];
            s = lh_run_spmv(ctx, tries[A->trie_slot], X->flat, X->flat_n, q->group[0].card, r);
        }
    } else if (exec == LH_EXEC_SPGEMM) {
        if (!is_spgemm(q, plan)) s = lh_fail(ctx, LH_EINVAL, "query is not an SpGEMM join-aggregate under this plan");
        else {
            // GROUP BY key implementation (Section 5): group_impl DENSE forces
            // the bitset + dense array wherever it fits, PRIVATE / SHARED keep
            // sort and hash, AUTO applies the density rule
            const uint32_t dm = q->group_impl == LH_GROUP_DENSE ? 2u : q->group_impl == LH_GROUP_AUTO ? 1u : 0u;
            s = lh_run_spgemm(ctx, tries[q->edges[0].trie_slot], tries[q->edges[1].trie_slot], r, dm);
        }
    } else {
        s = lh_run_generic(ctx, q, plan, tries, r, deadline_ms);
    }
    if (s != LH_OK) {
        for (void *p : r->allocs) lh_free(ctx, p);
        delete r;
        return s;
    }
    *out = r;
    return LH_OK;
}

extern "C" lh_status lh_join_aggregate(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan,
                                       lh_trie *const *tries, lh_result **out) {
    return lh_join_dispatch(ctx, q, plan, tries, out, 0.0);
}

extern "C" lh_status lh_result_wait(lh_ctx *ctx, lh_result *r, lh_result_view *v) {
    if (!ctx || !r || !v) return lh_fail(ctx, LH_EINVAL, "null argument");
    LH_TRY(lh_sync(ctx));
    memset(v, 0, sizeof(*v));
    v->exec = r->exec;
    if (r->hash_pending) {
        // compact the shared GROUP BY table into dense group arrays (slot order)
        r->hash_pending = false;
        uint32_t *flag = nullptr;
        uint64_t *pos = nullptr;
        uint64_t G = 0;
        lh_status s = lh_alloc(ctx, &flag, r->ht_cap);
        if (s == LH_OK) s = lh_alloc(ctx, &pos, (size_t)r->ht_cap + 1);
        if (s == LH_OK) {
            const unsigned g = lh_blocks(r->ht_cap, 256, (unsigned)ctx->num_sms * 8);
            LH_TRACED(ctx, "k_ht_flags", k_ht_flags<<<g, 256, 0, ctx->stream>>>(r->ht_tag, r->ht_cap, flag));
            s = lh_scan_u32_to_u64(ctx, flag, pos, r->ht_cap);
        }
        if (s == LH_OK) s = lh_readback(ctx, pos + r->ht_cap, sizeof(uint64_t), &G);
        if (s == LH_OK && G > 0xFFFFFFFFull) s = lh_fail(ctx, LH_EOVERFLOW, "too many groups");
        if (s == LH_OK) s = res_alloc(ctx, r, &r->group_keys, std::max<uint64_t>(1, G * r->n_group_cols));
        if (s == LH_OK) s = res_alloc(ctx, r, &r->d_gsum, std::max<uint64_t>(1, G));
        if (s == LH_OK) s = res_alloc(ctx, r, &r->d_gcount, std::max<uint64_t>(1, G));
        if (s == LH_OK && G) {
            HTab H{r->ht_tag, r->ht_keys, r->ht_sum, (unsigned long long *)r->ht_cnt, r->ht_cap};
            const unsigned g = lh_blocks(r->ht_cap, 256, (unsigned)ctx->num_sms * 8);
            LH_TRACED(ctx, "k_ht_scatter", k_ht_scatter<<<g, 256, 0, ctx->stream>>>(H, r->n_group_cols, pos, G, r->group_keys,
                                                                               r->d_gsum, r->d_gcount));
        }
        lh_free(ctx, flag);
        lh_free(ctx, pos);
        if (s == LH_OK) s = lh_sync(ctx);
        if (s != LH_OK) return s;
        r->ngroups = (uint32_t)G;
    }
    uint64_t cnt = 0, el[2] = {0, 0};
    if (r->d_count && r->d_elems == r->d_count + 1) {
        uint64_t w[3];
        LH_CU(cudaMemcpy(w, r->d_count, sizeof(w), cudaMemcpyDeviceToHost));
        cnt = w[0];
        el[0] = w[1];
        el[1] = w[2];
    } else {
        if (r->d_count) LH_CU(cudaMemcpy(&cnt, r->d_count, sizeof(cnt), cudaMemcpyDeviceToHost));
        if (r->d_elems) LH_CU(cudaMemcpy(el, r->d_elems, sizeof(el), cudaMemcpyDeviceToHost));
    }
    v->elements = el[0];
    v->visited = r->visited + el[1];
    v->count = cnt + r->host_count;
    if (r->ngroups) {
        std::vector<double> gs(r->ngroups);
        std::vector<uint64_t> gc(r->ngroups);
        LH_CU(cudaMemcpy(gs.data(), r->d_gsum, r->ngroups * sizeof(double), cudaMemcpyDeviceToHost));
        LH_CU(cudaMemcpy(gc.data(), r->d_gcount, r->ngroups * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        double s = 0.0;
        uint64_t c = 0;
        for (uint32_t g = 0; g < r->ngroups; ++g) { s += gs[g]; c += gc[g]; }
        v->sum = s;
        v->count = c;
    }
    v->ngroups = r->ngroups;
    v->n_group_cols = r->group_keys ? r->n_group_cols : 0;
    v->group_keys = r->group_keys;
    v->group_impl = r->group_impl;
    v->group_sum = r->d_gsum;
    v->group_count = r->d_gcount;
    v->nrows = r->nrows;
    v->y = r->y;
    if (r->nnz_pending) {
        LH_CU(cudaMemcpy(&r->nnz, r->c_off + r->nrows, sizeof(uint64_t), cudaMemcpyDeviceToHost));
        r->nnz_pending = false;
    }
    v->nnz = r->nnz;
    v->c_row = r->c_row;
    v->c_off = r->c_off;
    v->c_col = r->c_col;
    v->c_val = r->c_val;
    return LH_OK;
}

namespace {
// group totals -> (high, low) fp32 pair annotation columns
__global__ void k_split_pair(const double *sum, const uint64_t *cnt, uint32_t use_count, uint64_t n, float *hi,
                             float *lo) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double v = use_count ? (double)cnt[i] : sum[i];
        const float h = (float)v;
        hi[i] = h;
        lo[i] = (float)(v - (double)h);
    }
}
}  // namespace

extern "C" lh_status lh_join_to_trie(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan, lh_trie *const *tries,
                                     uint32_t n_out, const uint32_t *out_attrs, const lh_layout_policy *layout,
                                     lh_trie **out) {
    if (!ctx || !q || !plan || !out || (n_out && !out_attrs)) return lh_fail(ctx, LH_EINVAL, "null argument");
    *out = nullptr;
    if (n_out == 0 || n_out > LH_MAX_GROUP || n_out > LH_MAX_LEVELS)
        return lh_fail(ctx, LH_EINVAL, "1..%d output attributes", LH_MAX_LEVELS);
    lh_query q2 = *q;
    q2.n_group = n_out;
    for (uint32_t k = 0; k < n_out; ++k) {
        if (out_attrs[k] >= q->n_attrs) return lh_fail(ctx, LH_EINVAL, "output attribute out of range");
        q2.group[k] = lh_group{0, -1, out_attrs[k], 0};
    }
    const bool counts = q->semiring == LH_COUNT_U64;
    if (counts) q2.semiring = LH_SUM_F32_KAHAN;   // a tuple's weight: the number of join results under it
    if (q2.group_impl == LH_GROUP_DENSE) q2.group_impl = LH_GROUP_AUTO;
    if (q2.exec == LH_EXEC_AUTO) q2.exec = LH_EXEC_GENERIC;
    lh_result *r = nullptr;
    LH_TRY(lh_join_dispatch(ctx, &q2, plan, tries, &r, 0.0));
    lh_result_view v;
    lh_status s = lh_result_wait(ctx, r, &v);
    float *hi = nullptr, *lo = nullptr;
    const uint64_t G = v.ngroups;
    if (s == LH_OK && !v.group_keys) s = lh_fail(ctx, LH_EUNSUPPORTED, "the join did not produce key tuples");
    if (s == LH_OK) s = lh_alloc(ctx, &hi, std::max<uint64_t>(G, 1));
    if (s == LH_OK) s = lh_alloc(ctx, &lo, std::max<uint64_t>(G, 1));
    if (s == LH_OK && G) {
        const unsigned g = lh_blocks(G, 256, (unsigned)ctx->num_sms * 8);
        LH_TRACED(ctx, "k_split_pair", k_split_pair<<<g, 256, 0, ctx->stream>>>(v.group_sum, v.group_count, counts ? 1u : 0u,
                                                                           G, hi, lo));
    }
    if (s == LH_OK) {
        lh_relation_desc rel;
        memset(&rel, 0, sizeof(rel));
        rel.nrows = G;
        rel.nkeys = n_out;
        uint32_t order[LH_MAX_LEVELS];
        for (uint32_t k = 0; k < n_out; ++k) {
            rel.keys[k] = v.group_keys + (size_t)k * G;
            order[k] = k;
        }
        rel.nannos = 2;
        rel.annos[0] = hi;
        rel.annos[1] = lo;
        rel.anno_types[0] = rel.anno_types[1] = LH_T_F32;
        s = lh_build_trie(ctx, &rel, order, layout, LH_MERGE_FIRST, out);
    }
    if (s == LH_OK) s = lh_sync(ctx);   // the temporaries below are read by the build
    lh_free(ctx, hi);
    lh_free(ctx, lo);
    lh_result_free(ctx, r);
    return s;
}

extern "C" lh_status lh_result_free(lh_ctx *ctx, lh_result *r) {
    if (!ctx || !r) return LH_EINVAL;
    for (void *p : r->allocs) lh_free(ctx, p);
    delete r;
    return LH_OK;
}
