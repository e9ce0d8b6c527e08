// Batched uneven joins: thousands of independent triangle / 4-clique COUNT
// queries (Algorithm 1 unrolled for these two shapes over an oriented edge
// relation E(src < dst)) drained by ONE persistent launch.
//
// Work list: every first-level vertex a of every query's trie is an item; a
// vertex whose out-degree exceeds t_warp is split into items of `chunk`
// out-edges, so hubs of skewed graphs are spread over many warps.  Warps of a
// persistent grid (SMs x ctas_per_sm CTAs) claim items with an atomic ticket.
// For an item (a, edges [e0, e1)):
//   triangle: for each b in adj+(a)[e0, e1): |adj+(a) cap adj+(b)|
//   4-clique: for each such b and each c in adj+(a) cap adj+(b):
//             |{d in adj+(c) : d in adj+(a), d in adj+(b)}|
// Intersections are warp-cooperative: lanes walk the smaller set and probe
// the larger (a bitset probe where the trie chose the bitset layout, else a
// binary search).  The counter resets and the launch are captured once in a
// CUDA graph and replayed.  No kernel waits on another: the only shared state
// is the ticket counter.
#include <chrono>
#include <cmath>

#include "lh_join.cuh"

struct lh_batch {
    uint32_t n = 0;
    uint64_t *counts = nullptr;        // caller-owned
    DTrie *d_tries = nullptr;          // per query
    uint32_t *d_kind = nullptr;        // per query
    uint64_t *d_qoff = nullptr;        // first global vertex of each query (n + 1)
    uint64_t *d_item_off = nullptr;    // first item of each global vertex (V + 1)
    unsigned long long *d_ticket = nullptr;
    unsigned long long *d_elems = nullptr;  // input set elements of every executed intersection
    uint64_t n_vertices = 0, n_items = 0;
    lh_batch_tuning tuning{};
    unsigned grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kCBuf = 256;  // 4-clique: pending c values per warp

__device__ __forceinline__ uint64_t find_le(const uint64_t *off, uint64_t n, uint64_t x) {
    uint64_t lo = 0, hi = n;  // off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// items per vertex
__global__ void k_batch_items(const DTrie *tries, const uint64_t *qoff, uint32_t nq, uint64_t V, uint32_t t_warp,
                              uint32_t chunk, uint64_t *items) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t q = (uint32_t)find_le(qoff, nq, v);
        const DTrie &T = tries[q];
        const uint32_t p = (uint32_t)(v - qoff[q]);
        const uint32_t deg = T.lv[0].offs[p + 1] - T.lv[0].offs[p];
        items[v] = deg <= t_warp ? 1u : (deg + chunk - 1) / chunk;
    }
}

// count of x in the out-set of vertex u (level-1 set of u's first-level entry)
__device__ __forceinline__ bool in_adj(const DTrie &T, uint32_t pu, uint32_t lo, uint32_t hi, uint32_t x) {
    uint32_t pos;
    return lh_probe(T, 1, pu, lo, hi, x, &pos);
}

// Both shapes in one launch: each item reads its query's kind.
__global__ void __launch_bounds__(kThreads) k_batch(const DTrie *tries, const uint64_t *qoff, uint32_t nq,
                                                    uint64_t V, const uint64_t *item_off, uint32_t t_warp,
                                                    uint32_t chunk, unsigned long long *ticket,
                                                    unsigned long long *counts, const uint32_t *kinds,
                                                    unsigned long long *elems) {
    __shared__ uint32_t cbuf[kWarps][kCBuf];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t n_items = item_off[V];
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(ticket, 1ull);
        it = __shfl_sync(LH_FULL, it, 0);
        if (it >= n_items) break;
        const uint64_t v = find_le(item_off, V, it);
        const uint32_t q = (uint32_t)find_le(qoff, nq, v);
        const DTrie &T = tries[q];
        const uint32_t kind = kinds[q];
        const uint32_t pa = (uint32_t)(v - qoff[q]);
        const uint32_t a_lo = T.lv[0].offs[pa], a_hi = T.lv[0].offs[pa + 1];
        const uint32_t deg = a_hi - a_lo;
        uint32_t e0 = a_lo, e1 = a_hi;
        if (deg > t_warp) {
            const uint32_t c = (uint32_t)(it - item_off[v]);
            e0 = a_lo + c * chunk;
            e1 = min(a_hi, e0 + chunk);
        }
        unsigned long long local = 0, local_el = 0;  // local_el: warp-uniform
        for (uint32_t e = e0; e < e1; ++e) {
            const uint32_t b = __ldg(T.lv[1].vals + e);
            uint32_t pb;
            if (!lh_probe(T, 0, 0, 0, T.lv[0].n, b, &pb)) continue;  // b has no out-edges
            const uint32_t b_lo = __ldg(T.lv[0].offs + pb), b_hi = __ldg(T.lv[0].offs + pb + 1);
            // walk the smaller of adj+(a), adj+(b); probe the other
            const bool walk_a = (a_hi - a_lo) <= (b_hi - b_lo);
            const uint32_t w_lo = walk_a ? a_lo : b_lo, w_hi = walk_a ? a_hi : b_hi;
            const uint32_t o_p = walk_a ? pb : pa, o_lo = walk_a ? b_lo : a_lo, o_hi = walk_a ? b_hi : a_hi;
            local_el += (a_hi - a_lo) + (b_hi - b_lo);
            uint32_t nbuf = 0;
            for (uint32_t x0 = w_lo; x0 < w_hi; x0 += 32) {
                const uint32_t x = x0 + lane;
                bool hit = false;
                uint32_t cv = 0;
                if (x < w_hi) {
                    cv = __ldg(T.lv[1].vals + x);
                    hit = in_adj(T, o_p, o_lo, o_hi, cv);
                }
                if (kind == LH_BATCH_TRIANGLE) {
                    local += hit ? 1 : 0;
                    continue;
                }
                // 4-clique: stage the common neighbours c, expand them in batches
                const uint32_t ball = __ballot_sync(LH_FULL, hit);
                if (hit) cbuf[warp][nbuf + __popc(ball & ((1u << lane) - 1u))] = cv;
                nbuf += __popc(ball);
                __syncwarp();
                if (nbuf + 32 > kCBuf || x0 + 32 >= w_hi) {
                    for (uint32_t i = 0; i < nbuf; ++i) {
                        const uint32_t c = cbuf[warp][i];
                        uint32_t pc;
                        if (!lh_probe(T, 0, 0, 0, T.lv[0].n, c, &pc)) continue;
                        const uint32_t c_lo = __ldg(T.lv[0].offs + pc), c_hi = __ldg(T.lv[0].offs + pc + 1);
                        local_el += (c_hi - c_lo) + (a_hi - a_lo) + (b_hi - b_lo);
                        for (uint32_t y = c_lo + lane; y < c_hi; y += 32) {
                            const uint32_t d = __ldg(T.lv[1].vals + y);
                            if (in_adj(T, pa, a_lo, a_hi, d) && in_adj(T, pb, b_lo, b_hi, d)) ++local;
                        }
                    }
                    nbuf = 0;
                    __syncwarp();
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(LH_FULL, local, o);
        if (lane == 0 && local) atomicAdd(counts + q, local);
        if (lane == 0 && local_el) atomicAdd(elems, local_el);
    }
}

lh_status batch_build(lh_ctx *ctx, uint32_t n, const lh_batch_query *qs, const lh_batch_tuning &tun,
                      uint64_t *counts, lh_batch **out) {
    lh_batch *b = new lh_batch();
    b->n = n;
    b->counts = counts;
    b->tuning = tun;
    std::vector<DTrie> ht(n);
    std::vector<uint32_t> hk(n);
    std::vector<uint64_t> hq(n + 1, 0);
    lh_status s = LH_OK;
    for (uint32_t i = 0; i < n && s == LH_OK; ++i) {
        const lh_trie *t = qs[i].graph;
        if (!t || t->nlevels != 2 || t->key_order[0] != 0 || t->key_order[1] != 1)
            s = lh_fail(ctx, LH_EINVAL, "query %u: needs a 2-level edge trie with key order {0,1}", i);
        else if (qs[i].kind > LH_BATCH_CLIQUE4)
            s = lh_fail(ctx, LH_EINVAL, "query %u: unknown kind", i);
        else {
            ht[i] = lh_trie_dview(t);
            hk[i] = qs[i].kind;
            hq[i + 1] = hq[i] + t->lv[0].n;
        }
    }
    b->n_vertices = hq[n];
    auto fail = [&](lh_status st) {
        lh_free(ctx, b->d_tries); lh_free(ctx, b->d_kind); lh_free(ctx, b->d_qoff); lh_free(ctx, b->d_item_off);
        lh_free(ctx, b->d_ticket); lh_free(ctx, b->d_elems);
        delete b;
        return st;
    };
    if (s != LH_OK) return fail(s);
    if ((s = lh_alloc(ctx, &b->d_tries, n)) != LH_OK) return fail(s);
    if ((s = lh_alloc(ctx, &b->d_kind, n)) != LH_OK) return fail(s);
    if ((s = lh_alloc(ctx, &b->d_qoff, (size_t)n + 1)) != LH_OK) return fail(s);
    if ((s = lh_alloc(ctx, &b->d_item_off, b->n_vertices + 1)) != LH_OK) return fail(s);
    if ((s = lh_alloc(ctx, &b->d_ticket, 1)) != LH_OK) return fail(s);
    if ((s = lh_alloc(ctx, &b->d_elems, 1)) != LH_OK) return fail(s);
    cudaMemcpyAsync(b->d_tries, ht.data(), n * sizeof(DTrie), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(b->d_kind, hk.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(b->d_qoff, hq.data(), (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->stream);
    uint64_t *items = nullptr;
    if ((s = lh_alloc(ctx, &items, b->n_vertices)) != LH_OK) return fail(s);
    if (b->n_vertices)
        LH_TRACED(ctx, "k_batch_items", k_batch_items<<<lh_blocks(b->n_vertices, 256, (unsigned)ctx->num_sms * 8), 256, 0,
                                                    ctx->stream>>>(b->d_tries, b->d_qoff, n, b->n_vertices, tun.t_warp,
                                                                   tun.chunk, items));
    s = lh_scan_u64_to_u64(ctx, items, b->d_item_off, b->n_vertices);
    lh_free(ctx, items);
    if (s == LH_OK) s = lh_readback(ctx, b->d_item_off + b->n_vertices, sizeof(uint64_t), &b->n_items);
    if (s != LH_OK) return fail(s);
    b->grid = (unsigned)(ctx->num_sms * std::max<uint32_t>(1, tun.ctas_per_sm));
    // capture resets + the persistent launch (on a private stream: the
    // context stream may be the legacy default stream, which cannot capture)
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(counts, 0, n * sizeof(uint64_t), b->cap_stream);
        cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned long long), b->cap_stream);
        cudaMemsetAsync(b->d_elems, 0, sizeof(unsigned long long), b->cap_stream);
        k_batch<<<b->grid, kThreads, 0, b->cap_stream>>>(b->d_tries, b->d_qoff, n, b->n_vertices, b->d_item_off,
                                                             tun.t_warp, tun.chunk, b->d_ticket,
                                                             (unsigned long long *)counts, b->d_kind, b->d_elems);
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &b->graph);
        e = (e2 != cudaSuccess) ? e2 : cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (b->graph) cudaGraphDestroy(b->graph);
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        return fail(lh_fail(ctx, LH_ECUDA, "batch graph capture: %s", cudaGetErrorString(e)));
    }
    *out = b;
    return LH_OK;
}

}  // namespace

extern "C" lh_status lh_batch_create(lh_ctx *ctx, uint32_t n, const lh_batch_query *qs, const lh_batch_tuning *tuning,
                                     uint64_t *counts, lh_batch **out) {
    if (!ctx || !out || (n && (!qs || !counts))) return lh_fail(ctx, LH_EINVAL, "null argument");
    *out = nullptr;
    if (n == 0) return lh_fail(ctx, LH_EINVAL, "empty batch");
    lh_batch_tuning t = tuning ? *tuning : lh_batch_tuning{256, 256, 4, 0};
    if (t.chunk == 0 || t.t_warp == 0 || t.ctas_per_sm == 0 || t.ctas_per_sm > 32)
        return lh_fail(ctx, LH_EINVAL, "bad tuning");
    return batch_build(ctx, n, qs, t, counts, out);
}

extern "C" lh_status lh_batch_run(lh_ctx *ctx, lh_batch *b) {
    if (!ctx || !b) return LH_EINVAL;
    LhTraceScope scope(ctx, "k_batch");
    LH_CU(cudaGraphLaunch(b->exec, ctx->stream));
    return LH_OK;
}

extern "C" lh_status lh_batch_free(lh_ctx *ctx, lh_batch *b) {
    if (!ctx || !b) return LH_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    lh_free(ctx, b->d_tries); lh_free(ctx, b->d_kind); lh_free(ctx, b->d_qoff); lh_free(ctx, b->d_item_off);
    lh_free(ctx, b->d_ticket); lh_free(ctx, b->d_elems);
    delete b;
    return LH_OK;
}

extern "C" lh_status lh_batch_elements(lh_ctx *ctx, lh_batch *b, uint64_t *elements) {
    if (!ctx || !b || !elements) return lh_fail(ctx, LH_EINVAL, "null argument");
    return lh_readback(ctx, b->d_elems, sizeof(uint64_t), elements);
}

// Grid of tunings, successive halving: every candidate is timed once, the
// faster third is timed three more times, the best mean wins.  The timings
// run on a fixed sample of the batch -- every kTuneStride-th query (all of
// them for batches below 2 * kTuneStride) -- so the remaining queries are
// held out of the tuning and the full batch measures the chosen thresholds
// on mostly unseen work.
constexpr uint32_t kTuneStride = 4;

extern "C" lh_status lh_batch_autotune(lh_ctx *ctx, uint32_t n_all, const lh_batch_query *qs_all, uint64_t *counts,
                                       lh_batch_tuning *best, float *best_ms) {
    if (!ctx || !best) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (n_all == 0 || !qs_all || !counts) return lh_fail(ctx, LH_EINVAL, "empty batch");
    std::vector<lh_batch_query> sample;
    const uint32_t stride = n_all >= 2 * kTuneStride ? kTuneStride : 1u;
    for (uint32_t i = 0; i < n_all; i += stride) sample.push_back(qs_all[i]);
    const uint32_t n = (uint32_t)sample.size();
    const lh_batch_query *qs = sample.data();
    struct Cand { lh_batch_tuning t; double ms; int runs; };
    std::vector<Cand> cands;
    const uint32_t tw[] = {64, 256, 2048};
    const uint32_t ch[] = {32, 128, 512};
    const uint32_t cps[] = {2, 4, 8};
    for (uint32_t a : tw)
        for (uint32_t c : ch)
            for (uint32_t g : cps)
                if (c <= a) cands.push_back({lh_batch_tuning{a, c, g, 0}, 0.0, 0});
    cudaEvent_t e0, e1;
    LH_CU(cudaEventCreate(&e0));
    LH_CU(cudaEventCreate(&e1));
    lh_status s = LH_OK;
    auto time_one = [&](Cand &cd, int reps) -> lh_status {
        lh_batch *b = nullptr;
        LH_TRY(lh_batch_create(ctx, n, qs, &cd.t, counts, &b));
        LH_TRY(lh_batch_run(ctx, b));  // warm
        double tot = 0;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(e0, ctx->stream);
            lh_status st = lh_batch_run(ctx, b);
            cudaEventRecord(e1, ctx->stream);
            if (st != LH_OK) { lh_batch_free(ctx, b); return st; }
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        cd.ms = (cd.ms * cd.runs + tot) / (cd.runs + reps);
        cd.runs += reps;
        return lh_batch_free(ctx, b);
    };
    for (auto &cd : cands)
        if (s == LH_OK) s = time_one(cd, 1);
    if (s == LH_OK) {
        std::sort(cands.begin(), cands.end(), [](const Cand &x, const Cand &y) { return x.ms < y.ms; });
        const size_t keep = std::max<size_t>(1, cands.size() / 3);
        cands.resize(keep);
        for (auto &cd : cands)
            if (s == LH_OK) s = time_one(cd, 3);
        std::sort(cands.begin(), cands.end(), [](const Cand &x, const Cand &y) { return x.ms < y.ms; });
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != LH_OK) return s;
    *best = cands[0].t;
    if (best_ms) *best_ms = (float)cands[0].ms;
    return LH_OK;
}

// ------------------------------------------------- batched join-aggregate
// The batched form of lh_join_aggregate: queries whose shape the persistent
// kernel serves -- the triangle or 4-clique COUNT over one edge relation, in
// the identity attribute order, its trie built in key order {0, 1} -- go
// into one captured launch; the rest run through lh_join_aggregate.

namespace {

// 1: triangle, 2: 4-clique, 0: not a batch shape
uint32_t batch_shape(const lh_query &q, const lh_plan_t &p, lh_trie *const *tries, const lh_trie **graph) {
    if (q.semiring != LH_COUNT_U64 || q.n_group != 0) return 0;
    const uint32_t k = q.n_attrs;
    if (!((k == 3 && q.n_edges == 3) || (k == 4 && q.n_edges == 6))) return 0;
    if (p.n_attrs != k) return 0;
    for (uint32_t i = 0; i < k; ++i)
        if (p.order[i] != i) return 0;
    const int32_t slot = q.edges[0].trie_slot;
    if (slot < 0 || !tries || !tries[slot]) return 0;
    uint32_t seen = 0;   // bit (a * 4 + b) for pattern edge (a, b), a < b
    for (uint32_t e = 0; e < q.n_edges; ++e) {
        const lh_edge &E = q.edges[e];
        if (E.trie_slot != slot || E.nattrs != 2 || E.flat) return 0;
        const uint32_t a = E.attrs[0], b = E.attrs[1];
        if (a >= b || b >= k) return 0;
        seen |= 1u << (a * 4 + b);
    }
    uint32_t want = 0;
    for (uint32_t a = 0; a < k; ++a)
        for (uint32_t b = a + 1; b < k; ++b) want |= 1u << (a * 4 + b);
    if (seen != want) return 0;
    const lh_trie *t = tries[slot];
    if (t->nlevels != 2 || t->key_order[0] != 0 || t->key_order[1] != 1) return 0;
    *graph = t;
    return k == 3 ? 1u : 2u;
}

}  // namespace

extern "C" lh_status lh_join_aggregate_batch(lh_ctx *ctx, uint32_t n, const lh_query *qs, const lh_plan_t *plans,
                                             lh_trie *const *const *tries, const lh_batch_tuning *tuning,
                                             lh_result **out) {
    if (!ctx) return LH_EINVAL;
    if (n && (!qs || !plans || !tries || !out)) return lh_fail(ctx, LH_EINVAL, "null argument");
    for (uint32_t i = 0; i < n; ++i) out[i] = nullptr;
    std::vector<lh_batch_query> bq;
    std::vector<uint32_t> bidx;
    for (uint32_t i = 0; i < n; ++i) {
        const lh_trie *g = nullptr;
        const uint32_t shape = batch_shape(qs[i], plans[i], tries[i], &g);
        if (shape) {
            bq.push_back(lh_batch_query{shape == 1 ? (uint32_t)LH_BATCH_TRIANGLE : (uint32_t)LH_BATCH_CLIQUE4, g});
            bidx.push_back(i);
        }
    }
    auto fail = [&](lh_status st) {
        for (uint32_t i = 0; i < n; ++i)
            if (out[i]) {
                lh_result_free(ctx, out[i]);
                out[i] = nullptr;
            }
        return st;
    };
    // the shapes the persistent kernel serves: one launch, one readback
    if (!bq.empty()) {
        const uint32_t nb = (uint32_t)bq.size();
        uint64_t *counts = nullptr;
        lh_batch *b = nullptr;
        lh_status s = lh_alloc(ctx, &counts, nb);
        if (s == LH_OK) s = lh_batch_create(ctx, nb, bq.data(), tuning, counts, &b);
        if (s == LH_OK) s = lh_batch_run(ctx, b);
        std::vector<uint64_t> hc(nb, 0);
        if (s == LH_OK) {
            cudaError_t e = cudaMemcpyAsync(hc.data(), counts, nb * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "batch counts: %s", cudaGetErrorString(e));
        }
        if (s == LH_OK) s = lh_sync(ctx);
        if (b) lh_batch_free(ctx, b);
        lh_free(ctx, counts);
        if (s != LH_OK) return fail(s);
        for (uint32_t j = 0; j < nb; ++j) {
            lh_result *r = new lh_result();
            r->exec = LH_EXEC_GENERIC;
            r->semiring = LH_COUNT_U64;
            r->host_count = hc[j];
            out[bidx[j]] = r;
        }
    }
    // every other query through the generic entry point
    for (uint32_t i = 0; i < n; ++i) {
        if (out[i]) continue;
        lh_status s = lh_join_aggregate(ctx, &qs[i], &plans[i], tries[i], &out[i]);
        if (s != LH_OK) return fail(s);
    }
    return LH_OK;
}
