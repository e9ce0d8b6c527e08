// Learned planner (no paper counterpart; it replaces the hand-set icost and
// weight tables of Section 4 with a model trained on the engine's own
// timings) and the exhaustive judge.
//
//   features  per (query, attribute order, layout policy), from device-side
//             statistics of the tries that order needs: relation sizes; per
//             attribute position the log2 set-size median, 90th percentile
//             and maximum and the density of its trie level, and the Section
//             4 cost term log2(1 + icost x weight); the order as a position
//             one-hot; the layout one-hot.
//   model     MLP n_in -> H -> H -> 1 (ReLU), fp32, predicting log(ms);
//             forward, backward (mean squared error) and Adam are this
//             file's kernels, in a fixed summation order.
//   LEARNED   scores every candidate (order x layout policy) and keeps the
//             lowest prediction.
//   EXHAUSTIVE builds, runs and times every candidate with a per-candidate
//             host-side time budget and keeps the fastest.
#include <chrono>
#include <cmath>
#include <random>

#include "lh_join.cuh"
#include "lh_plan.cuh"

struct lh_model {
    uint32_t n_in = 0, hidden = 0;
    uint64_t n_params = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    uint32_t step = 0;
    // forward / backward scratch, sized for `cap` samples
    uint32_t cap = 0;
    float *z1 = nullptr, *z2 = nullptr, *out = nullptr, *dout = nullptr, *dz1 = nullptr, *dz2 = nullptr;
    float *loss = nullptr;
};

namespace {

struct Layout {
    uint64_t w1, b1, w2, b2, w3, b3, total;
};

Layout layout_of(uint32_t n_in, uint32_t H) {
    Layout L;
    L.w1 = 0;
    L.b1 = L.w1 + (uint64_t)n_in * H;
    L.w2 = L.b1 + H;
    L.b2 = L.w2 + (uint64_t)H * H;
    L.w3 = L.b2 + H;
    L.b3 = L.w3 + H;
    L.total = L.b3 + 1;
    return L;
}

// out[i][o] = b[o] + sum_k in[i][k] W[k][o]  (optionally through ReLU)
__global__ void k_mlp_layer(const float *in, uint32_t n, uint32_t din, const float *W, const float *b, uint32_t dout,
                            float *z) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * dout) return;
    const uint32_t i = (uint32_t)(t / dout), o = (uint32_t)(t % dout);
    float acc = b[o];
    for (uint32_t k = 0; k < din; ++k) acc = fmaf(in[(uint64_t)i * din + k], W[(uint64_t)k * dout + o], acc);
    z[t] = acc;
}

__global__ void k_relu_copy(const float *z, uint64_t n, float *h) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) h[t] = fmaxf(z[t], 0.f);
}

// layers with ReLU inputs read z and apply the ReLU on the fly
__global__ void k_mlp_layer_relu_in(const float *zin, uint32_t n, uint32_t din, const float *W, const float *b,
                                    uint32_t dout, float *z) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * dout) return;
    const uint32_t i = (uint32_t)(t / dout), o = (uint32_t)(t % dout);
    float acc = b[o];
    for (uint32_t k = 0; k < din; ++k) acc = fmaf(fmaxf(zin[(uint64_t)i * din + k], 0.f), W[(uint64_t)k * dout + o], acc);
    z[t] = acc;
}

// d_out = 2/n (out - y); loss = mean (out - y)^2 (one block, fixed order)
__global__ void k_mse(const float *out, const float *y, uint32_t n, float *dout, float *loss) {
    __shared__ float part[256];
    float s = 0.f;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float r = out[i] - y[i];
        dout[i] = 2.f * r / (float)n;
        s = fmaf(r, r, s);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (uint32_t w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)n;
}

// dW[k][o] = sum_i act(in[i][k]) dz[i][o]; db[o] = sum_i dz[i][o]
__global__ void k_mlp_wgrad(const float *in, uint32_t relu_in, const float *dz, uint32_t n, uint32_t din,
                            uint32_t dout, float *dW, float *db) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (uint64_t)din * dout) {
        const uint32_t k = (uint32_t)(t / dout), o = (uint32_t)(t % dout);
        float acc = 0.f;
        for (uint32_t i = 0; i < n; ++i) {
            float a = in[(uint64_t)i * din + k];
            if (relu_in) a = fmaxf(a, 0.f);
            acc = fmaf(a, dz[(uint64_t)i * dout + o], acc);
        }
        dW[t] = acc;
    } else if (t < (uint64_t)din * dout + dout) {
        const uint32_t o = (uint32_t)(t - (uint64_t)din * dout);
        float acc = 0.f;
        for (uint32_t i = 0; i < n; ++i) acc += dz[(uint64_t)i * dout + o];
        db[o] = acc;
    }
}

// dz_prev[i][k] = (sum_o dz[i][o] W[k][o]) * (z_prev[i][k] > 0)
__global__ void k_mlp_back(const float *dz, const float *W, const float *zprev, uint32_t n, uint32_t din,
                           uint32_t dout, float *dzprev) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * din) return;
    const uint32_t i = (uint32_t)(t / din), k = (uint32_t)(t % din);
    float acc = 0.f;
    for (uint32_t o = 0; o < dout; ++o) acc = fmaf(dz[(uint64_t)i * dout + o], W[(uint64_t)k * dout + o], acc);
    dzprev[t] = zprev[t] > 0.f ? acc : 0.f;
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, uint64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gg = g[t];
    const float mm = b1 * m[t] + (1.f - b1) * gg;
    const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    p[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void k_gather_rows(const float *X, const float *y, const uint32_t *idx, uint32_t n, uint32_t d, float *Xo,
                              float *yo) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)n * d) return;
    const uint32_t i = (uint32_t)(t / d), k = (uint32_t)(t % d);
    Xo[t] = X[(uint64_t)idx[i] * d + k];
    if (k == 0) yo[i] = y[idx[i]];
}

unsigned blocks_for(uint64_t n) { return (unsigned)((n + 255) / 256); }

lh_status ensure_cap(lh_ctx *ctx, lh_model *m, uint32_t n) {
    if (n <= m->cap) return LH_OK;
    m->cap = 0;   // until every buffer is reallocated: a failure here leaves none usable
    float **bufs[] = {&m->z1, &m->z2, &m->dz1, &m->dz2};
    for (float **b : bufs) {
        lh_free(ctx, *b);
        LH_TRY(lh_alloc(ctx, b, (size_t)n * m->hidden));
    }
    lh_free(ctx, m->out);
    lh_free(ctx, m->dout);
    LH_TRY(lh_alloc(ctx, &m->out, n));
    LH_TRY(lh_alloc(ctx, &m->dout, n));
    m->cap = n;
    return LH_OK;
}

lh_status forward(lh_ctx *ctx, const lh_model *mc, const float *X, uint32_t n, float *out) {
    lh_model *m = const_cast<lh_model *>(mc);
    LH_TRY(ensure_cap(ctx, m, n));
    const Layout L = layout_of(m->n_in, m->hidden);
    const uint32_t H = m->hidden;
    const float *P = m->params;
    LH_TRACED(ctx, "k_mlp_layer", k_mlp_layer<<<blocks_for((uint64_t)n * H), 256, 0, ctx->stream>>>(X, n, m->n_in, P + L.w1, P + L.b1, H, m->z1));
    LH_TRACED(ctx, "k_mlp_layer", k_mlp_layer_relu_in<<<blocks_for((uint64_t)n * H), 256, 0, ctx->stream>>>(m->z1, n, H, P + L.w2, P + L.b2, H, m->z2));
    LH_TRACED(ctx, "k_mlp_layer", k_mlp_layer_relu_in<<<blocks_for(n), 256, 0, ctx->stream>>>(m->z2, n, H, P + L.w3, P + L.b3, 1, out));
    LH_LAUNCH_CHECK();
    return LH_OK;
}

lh_status loss_grad(lh_ctx *ctx, lh_model *m, const float *X, const float *y, uint32_t n, float *loss) {
    // size the scratch first: m->out may not exist before this call
    LH_TRY(ensure_cap(ctx, m, n));
    LH_TRY(forward(ctx, m, X, n, m->out));
    const Layout L = layout_of(m->n_in, m->hidden);
    const uint32_t H = m->hidden;
    float *P = m->params, *G = m->grads;
    LH_TRACED(ctx, "k_mse", k_mse<<<1, 256, 0, ctx->stream>>>(m->out, y, n, m->dout, loss));
    // layer 3: dW3 = h2^T dout, db3 = sum dout
    LH_TRACED(ctx, "k_mlp_wgrad", k_mlp_wgrad<<<blocks_for(H + 1), 256, 0, ctx->stream>>>(m->z2, 1, m->dout, n, H, 1, G + L.w3, G + L.b3));
    LH_TRACED(ctx, "k_mlp_back", k_mlp_back<<<blocks_for((uint64_t)n * H), 256, 0, ctx->stream>>>(m->dout, P + L.w3, m->z2, n, H, 1, m->dz2));
    LH_TRACED(ctx, "k_mlp_wgrad", k_mlp_wgrad<<<blocks_for((uint64_t)H * H + H), 256, 0, ctx->stream>>>(m->z1, 1, m->dz2, n, H, H, G + L.w2, G + L.b2));
    LH_TRACED(ctx, "k_mlp_back", k_mlp_back<<<blocks_for((uint64_t)n * H), 256, 0, ctx->stream>>>(m->dz2, P + L.w2, m->z1, n, H, H, m->dz1));
    LH_TRACED(ctx, "k_mlp_wgrad", k_mlp_wgrad<<<blocks_for((uint64_t)m->n_in * H + H), 256, 0, ctx->stream>>>(X, 0, m->dz1, n, m->n_in, H, G + L.w1, G + L.b1));
    LH_LAUNCH_CHECK();
    return LH_OK;
}

lh_status adam(lh_ctx *ctx, lh_model *m, float lr, float b1, float b2, float eps) {
    m->step += 1;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    LH_TRACED(ctx, "k_adam", k_adam<<<blocks_for(m->n_params), 256, 0, ctx->stream>>>(m->params, m->grads, m->m, m->v, m->n_params, lr, b1, b2, eps, c1, c2));
    LH_LAUNCH_CHECK();
    return LH_OK;
}

// ------------------------------------------------------- trie level stats

// histogram of floor(log2(set size)) over the sets of one level, and the
// summed value span (max - min + 1) of those sets
__global__ void k_level_stats(const uint32_t *vals, const uint32_t *poffs, uint64_t nsets, uint32_t n0,
                              unsigned long long *hist, unsigned long long *span) {
    __shared__ unsigned long long h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long sp = 0;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsets; s += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t lo = poffs ? poffs[s] : 0, hi = poffs ? poffs[s + 1] : n0;
        if (hi <= lo) continue;
        atomicAdd(&h[31 - __clz(hi - lo)], 1ull);
        sp += (unsigned long long)(vals[hi - 1] - vals[lo]) + 1ull;
    }
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(LH_FULL, sp, o);
    if ((threadIdx.x & 31) == 0 && sp) atomicAdd(span, sp);
}

struct LevelStats {
    float q50, q90, q99, qmax, density;
};

lh_status level_stats(lh_ctx *ctx, const lh_trie *t, uint32_t l, LevelStats *out) {
    const TrieLevel &L = t->lv[l];
    const uint64_t nsets = (l == 0) ? 1 : t->lv[l - 1].n;
    const uint32_t *poffs = (l == 0) ? nullptr : t->lv[l - 1].offs;
    unsigned long long *buf = nullptr;
    LH_TRY(lh_alloc(ctx, &buf, 34));
    LH_CU(cudaMemsetAsync(buf, 0, 34 * sizeof(unsigned long long), ctx->stream));
    if (L.n)
        LH_TRACED(ctx, "k_level_stats", k_level_stats<<<lh_blocks(nsets, 256, (unsigned)ctx->num_sms * 4), 256, 0, ctx->stream>>>(
                                            L.vals, poffs, nsets, (uint32_t)L.n, buf, buf + 33));
    unsigned long long h[34];
    lh_status s = lh_readback(ctx, buf, sizeof(h), h);
    lh_free(ctx, buf);
    LH_TRY(s);
    uint64_t tot = 0;
    for (int b = 0; b < 33; ++b) tot += h[b];
    auto q = [&](double frac) -> float {
        if (!tot) return 0.f;
        const uint64_t want = (uint64_t)std::ceil(frac * (double)tot);
        uint64_t acc = 0;
        for (int b = 0; b < 33; ++b) {
            acc += h[b];
            if (acc >= want) return (float)b;
        }
        return 32.f;
    };
    out->q50 = q(0.5);
    out->q90 = q(0.9);
    out->q99 = q(0.99);
    out->qmax = q(1.0);
    out->density = h[33] ? (float)((double)L.n / (double)h[33]) : 0.f;
    return LH_OK;
}

int policy_index(uint32_t ratio) {
    switch (ratio) {
        case 0: return 0;
        case 8: return 1;
        case 32: return 2;
        default: return 3;
    }
}

lh_status features(lh_ctx *ctx, const lh_query *q, const uint32_t *order, uint32_t ratio0, uint32_t ratio_inner,
                   const lh_trie *const *edge_tries, float *f) {
    for (int i = 0; i < LH_NFEAT; ++i) f[i] = 0.f;
    uint64_t cards[LH_MAX_EDGES];
    for (uint32_t e = 0; e < q->n_edges; ++e) {
        uint64_t card = q->edges[e].card;
        const lh_trie *t = edge_tries[e];
        if (t) card = t->lv[t->nlevels - 1].n;
        else if (!card) card = q->edges[e].flat_n;
        cards[e] = card ? card : 1;
        if (e < 6) f[e] = (float)std::log2((double)card + 1.0);
    }
    // the Section 4 cost model's term of each attribute, as a prior
    int64_t w[LH_MAX_ATTRS] = {0};
    lh_weights(q, cards, w);
    for (uint32_t d = 0; d < q->n_attrs && d < 5; ++d) {
        const uint32_t v = order[d];
        LevelStats best{1e30f, 1e30f, 1e30f, 1e30f, 0.f};
        bool any = false;
        for (uint32_t e = 0; e < q->n_edges; ++e) {
            const lh_trie *t = edge_tries[e];
            if (!t) continue;
            for (uint32_t l = 0; l < t->nlevels; ++l) {
                if (q->edges[e].attrs[t->key_order[l]] != v) continue;
                LevelStats st;
                LH_TRY(level_stats(ctx, t, l, &st));
                best.q50 = std::min(best.q50, st.q50);
                best.q90 = std::min(best.q90, st.q90);
                best.q99 = std::min(best.q99, st.q99);
                best.qmax = std::min(best.qmax, st.qmax);
                best.density = std::max(best.density, st.density);
                any = true;
            }
        }
        if (any) {
            float *g = f + 6 + 5 * d;
            g[0] = best.q50;
            g[1] = best.q90;
            g[2] = best.qmax;
            g[3] = best.density;
        }
        f[6 + 5 * d + 4] = (float)std::log2(1.0 + (double)lh_icost_vertex(q, order, d) * (double)w[v]);
        if (v < 5) f[31 + 5 * d + v] = 1.f;
    }
    f[56 + policy_index(ratio0)] = 1.f;
    f[60 + policy_index(ratio_inner)] = 1.f;
    return LH_OK;
}

// ------------------------------------------------------------ trie cache

// annotation merge a relation's columns allow: float columns sum, a
// (price, discount) pair forms its expression, anything else keeps the first
lh_merge merge_for(const lh_relation_desc *rel) {
    if (rel->nannos == 2 && rel->anno_types[1] == LH_T_I8 &&
        (rel->anno_types[0] == LH_T_F64 || rel->anno_types[0] == LH_T_F32))
        return LH_MERGE_PRICE_DISCOUNT;
    for (uint32_t c = 0; c < rel->nannos; ++c)
        if (rel->anno_types[c] != LH_T_F32 && rel->anno_types[c] != LH_T_F64) return LH_MERGE_FIRST;
    return LH_MERGE_SUM;
}

// a candidate layout: ratio of level 0 and of the deeper levels
struct Pol {
    uint32_t r0, r1;
};

lh_layout_policy policy_of(Pol p) {
    lh_layout_policy pol{};
    pol.bs_ratio = p.r0;
    pol.bs_min_card = (p.r0 || p.r1) ? 32u : 0u;
    pol.per_level = 1;
    pol.level_ratio[0] = p.r0;
    for (int l = 1; l < LH_MAX_LEVELS; ++l) pol.level_ratio[l] = p.r1;
    return pol;
}

std::vector<Pol> candidate_policies(const lh_plan_opts *o) {
    std::vector<Pol> out;
    for (uint32_t i = 0; i < o->n_policies; ++i) {
        if (!o->per_level) {
            out.push_back({o->policies[i], o->policies[i]});
            continue;
        }
        for (uint32_t j = 0; j < o->n_policies; ++j) out.push_back({o->policies[i], o->policies[j]});
    }
    return out;
}

struct TrieKey {
    const lh_relation_desc *rel;
    uint32_t order[LH_MAX_LEVELS];
    uint32_t r0, r1;
    bool operator<(const TrieKey &o) const {
        if (rel != o.rel) return rel < o.rel;
        if (r0 != o.r0) return r0 < o.r0;
        if (r1 != o.r1) return r1 < o.r1;
        return memcmp(order, o.order, sizeof(order)) < 0;
    }
};

struct TrieCache {
    lh_ctx *ctx;
    std::map<TrieKey, lh_trie *> tries;
    ~TrieCache() {
        for (auto &kv : tries) lh_trie_free(ctx, kv.second);
    }
    lh_status get(const lh_relation_desc *rel, const uint32_t *ko, uint32_t nk, Pol p, lh_trie **out) {
        TrieKey k;
        memset(&k, 0, sizeof(k));
        k.rel = rel;
        k.r0 = p.r0;
        k.r1 = p.r1;
        for (uint32_t i = 0; i < nk; ++i) k.order[i] = ko[i];
        auto it = tries.find(k);
        if (it != tries.end()) {
            *out = it->second;
            return LH_OK;
        }
        const lh_layout_policy pol = policy_of(p);
        lh_trie *t = nullptr;
        LH_TRY(lh_build_trie(ctx, rel, ko, &pol, merge_for(rel), &t));
        tries[k] = t;
        *out = t;
        return LH_OK;
    }
};

// tries of every edge of q under `order` (flat edges: null)
lh_status edge_tries_for(TrieCache &cache, const lh_query *q, const lh_relation_desc *const *rels,
                         const uint32_t *order, Pol pol, lh_trie **tries) {
    for (uint32_t e = 0; e < q->n_edges; ++e) {
        tries[e] = nullptr;
        if (q->edges[e].trie_slot < 0) continue;
        if (!rels[e]) return lh_fail(cache.ctx, LH_EINVAL, "edge %u: no relation", e);
        uint32_t ko[LH_MAX_LEVELS];
        if (!lh_key_order_for(q, order, q->n_attrs, e, ko)) return lh_fail(cache.ctx, LH_EINVAL, "edge %u: key order", e);
        LH_TRY(cache.get(rels[e], ko, q->edges[e].nattrs, pol, &tries[e]));
    }
    return LH_OK;
}

// query copy whose edges point at slot e of the per-edge trie array
lh_query with_edge_slots(const lh_query *q) {
    lh_query r = *q;
    for (uint32_t e = 0; e < q->n_edges; ++e)
        if (r.edges[e].trie_slot >= 0) r.edges[e].trie_slot = (int32_t)e;
    return r;
}

}  // namespace

lh_status lh_join_dispatch(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan, lh_trie *const *tries,
                           lh_result **out, double deadline_ms);

// ----------------------------------------------------------------- planners

lh_status lh_plan_learned(lh_ctx *ctx, const lh_query *q, const lh_model *model, const lh_relation_desc *const *rels,
                          const lh_plan_opts *o, const uint64_t *cards, lh_plan_t *out) {
    (void)cards;
    if (model->n_in != LH_NFEAT) return lh_fail(ctx, LH_EINVAL, "model input width %u != %d", model->n_in, LH_NFEAT);
    std::vector<std::vector<uint32_t>> orders;
    lh_candidate_orders(q, orders);
    TrieCache cache{ctx, {}};
    std::vector<float> feats;
    const std::vector<Pol> pols = candidate_policies(o);
    std::vector<std::pair<size_t, Pol>> cand;
    for (size_t i = 0; i < orders.size(); ++i) {
        lh_trie *tr[LH_MAX_EDGES];
        LH_TRY(edge_tries_for(cache, q, rels, orders[i].data(), Pol{0, 0}, tr));
        for (const Pol &pl : pols) {
            float f[LH_NFEAT];
            LH_TRY(features(ctx, q, orders[i].data(), pl.r0, pl.r1, tr, f));
            feats.insert(feats.end(), f, f + LH_NFEAT);
            cand.push_back({i, pl});
        }
    }
    const uint32_t nc = (uint32_t)cand.size();
    float *dX = nullptr, *dY = nullptr;
    LH_TRY(lh_alloc(ctx, &dX, feats.size()));
    lh_status s = lh_alloc(ctx, &dY, nc);
    if (s == LH_OK) {
        cudaMemcpyAsync(dX, feats.data(), feats.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
        s = forward(ctx, model, dX, nc, dY);
    }
    std::vector<float> pred(nc);
    if (s == LH_OK) {
        cudaMemcpyAsync(pred.data(), dY, nc * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "learned planner sync");
    }
    lh_free(ctx, dX);
    lh_free(ctx, dY);
    LH_TRY(s);
    uint32_t best = 0;
    for (uint32_t c = 1; c < nc; ++c)
        if (pred[c] < pred[best]) best = c;
    int64_t w[LH_MAX_ATTRS] = {0};
    lh_weights(q, cards, w);
    const auto &bo = orders[cand[best].first];
    for (uint32_t i = 0; i < q->n_attrs; ++i) out->order[i] = bo[i];
    out->bs_ratio = cand[best].second.r0;
    out->bs_ratio_inner = cand[best].second.r1;
    out->exec = lh_exec_for(q, out->order);
    out->cost = lh_cost_of(q, out->order, w);
    out->predicted_log_ms = pred[best];
    out->n_candidates = nc;
    return LH_OK;
}

lh_status lh_plan_exhaustive(lh_ctx *ctx, const lh_query *q, const lh_relation_desc *const *rels,
                             const lh_plan_opts *o, lh_plan_t *out) {
    std::vector<std::vector<uint32_t>> orders;
    lh_candidate_orders(q, orders);
    // candidates in the order of the Section 4 cost estimate, so that fast
    // plans come early; each later run is cut once it takes 1.25x the best
    // time seen so far (it cannot be the fastest), which keeps the search
    // exhaustive while bounding the time spent on hopeless plans
    {
        uint64_t cards[LH_MAX_EDGES];
        for (uint32_t e = 0; e < q->n_edges; ++e) {
            uint64_t c = q->edges[e].card;
            if (!c && q->edges[e].trie_slot < 0) c = q->edges[e].flat_n;
            if (!c && rels && rels[e]) c = rels[e]->nrows;
            cards[e] = c ? c : 1;
        }
        int64_t w[LH_MAX_ATTRS] = {0};
        lh_weights(q, cards, w);
        std::stable_sort(orders.begin(), orders.end(), [&](const std::vector<uint32_t> &x, const std::vector<uint32_t> &y) {
            return lh_cost_of(q, x.data(), w) < lh_cost_of(q, y.data(), w);
        });
    }
    TrieCache cache{ctx, {}};
    const lh_query qs = with_edge_slots(q);
    cudaEvent_t e0, e1;
    LH_CU(cudaEventCreate(&e0));
    LH_CU(cudaEventCreate(&e1));
    double best_ms = 1e300;
    size_t best_i = 0;
    Pol best_pol{0, 0};
    uint32_t n = 0;
    lh_status s = LH_OK;
    const double budget = o->time_budget_ms > 0 ? o->time_budget_ms : 0.0;
    const std::vector<Pol> pols = candidate_policies(o);
    for (size_t i = 0; i < orders.size() && s == LH_OK; ++i) {
        for (size_t pi = 0; pi < pols.size() && s == LH_OK; ++pi) {
            lh_trie *tr[LH_MAX_EDGES];
            s = edge_tries_for(cache, q, rels, orders[i].data(), pols[pi], tr);
            if (s != LH_OK) break;
            lh_plan_t p = *out;
            for (uint32_t k = 0; k < q->n_attrs; ++k) p.order[k] = orders[i][k];
            p.bs_ratio = pols[pi].r0;
            p.bs_ratio_inner = pols[pi].r1;
            p.exec = LH_EXEC_AUTO;
            double tot = 0;
            bool timed_out = false;
            const uint32_t reps = std::max<uint32_t>(1, o->repeats);
            double cut = budget;
            if (best_ms < 1e299) cut = cut > 0 ? std::min(cut, 1.25 * best_ms) : 1.25 * best_ms;
            for (uint32_t r = 0; r <= reps; ++r) {  // first run warms up
                lh_result *res = nullptr;
                cudaEventRecord(e0, ctx->stream);
                lh_status st = lh_join_dispatch(ctx, &qs, &p, tr, &res, cut);
                cudaEventRecord(e1, ctx->stream);
                if (st == LH_ETIMEOUT) {
                    timed_out = true;
                    break;
                }
                if (st != LH_OK) { s = st; break; }
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                lh_result_free(ctx, res);
                if (r > 0) tot += ms;
            }
            if (s != LH_OK) break;
            ++n;
            const double ms = timed_out ? 1e299 : tot / reps;
            if (ms < best_ms) {
                best_ms = ms;
                best_i = i;
                best_pol = pols[pi];
            }
        }
    }
    cudaStreamSynchronize(ctx->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LH_TRY(s);
    for (uint32_t k = 0; k < q->n_attrs; ++k) out->order[k] = orders[best_i][k];
    out->bs_ratio = best_pol.r0;
    out->bs_ratio_inner = best_pol.r1;
    out->exec = lh_exec_for(q, out->order);
    out->measured_ms = (float)best_ms;
    out->n_candidates = n;
    return LH_OK;
}

// -------------------------------------------------------------------- C ABI

extern "C" lh_status lh_model_create(lh_ctx *ctx, uint32_t n_in, uint32_t hidden, uint64_t seed, lh_model **out) {
    if (!ctx || !out || n_in == 0 || hidden == 0 || hidden > 1024) return lh_fail(ctx, LH_EINVAL, "bad model shape");
    lh_model *m = new lh_model();
    m->n_in = n_in;
    m->hidden = hidden;
    const Layout L = layout_of(n_in, hidden);
    m->n_params = L.total;
    std::vector<float> p(L.total, 0.f);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    auto glorot = [&](uint64_t at, uint32_t a, uint32_t b) {
        const double s = std::sqrt(6.0 / (a + b));
        for (uint64_t i = 0; i < (uint64_t)a * b; ++i) p[at + i] = (float)(U(rng) * s);
    };
    glorot(L.w1, n_in, hidden);
    glorot(L.w2, hidden, hidden);
    glorot(L.w3, hidden, 1);
    lh_status s = lh_alloc(ctx, &m->params, L.total);
    if (s == LH_OK) s = lh_alloc(ctx, &m->grads, L.total);
    if (s == LH_OK) s = lh_alloc(ctx, &m->m, L.total);
    if (s == LH_OK) s = lh_alloc(ctx, &m->v, L.total);
    if (s == LH_OK) s = lh_alloc(ctx, &m->loss, 1);
    if (s == LH_OK) {
        cudaMemcpyAsync(m->params, p.data(), L.total * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
        cudaMemsetAsync(m->grads, 0, L.total * sizeof(float), ctx->stream);
        cudaMemsetAsync(m->m, 0, L.total * sizeof(float), ctx->stream);
        cudaMemsetAsync(m->v, 0, L.total * sizeof(float), ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "model init");
    }
    if (s != LH_OK) {
        lh_model_free(ctx, m);
        return s;
    }
    *out = m;
    return LH_OK;
}

extern "C" lh_status lh_model_free(lh_ctx *ctx, lh_model *m) {
    if (!ctx || !m) return LH_EINVAL;
    float *bufs[] = {m->params, m->grads, m->m, m->v, m->z1, m->z2, m->out, m->dout, m->dz1, m->dz2, m->loss};
    for (float *b : bufs) lh_free(ctx, b);
    delete m;
    return LH_OK;
}

extern "C" lh_status lh_model_buffers(lh_ctx *ctx, lh_model *m, float **params, float **grads, uint64_t *n) {
    if (!ctx || !m) return LH_EINVAL;
    if (params) *params = m->params;
    if (grads) *grads = m->grads;
    if (n) *n = m->n_params;
    return LH_OK;
}

extern "C" lh_status lh_model_forward(lh_ctx *ctx, const lh_model *m, const float *X, uint32_t n, float *out) {
    if (!ctx || !m || (n && (!X || !out))) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (!n) return LH_OK;
    return forward(ctx, m, X, n, out);
}

extern "C" lh_status lh_model_loss_grad(lh_ctx *ctx, lh_model *m, const float *X, const float *y, uint32_t n,
                                        float *loss) {
    if (!ctx || !m || !X || !y || !loss || n == 0) return lh_fail(ctx, LH_EINVAL, "bad argument");
    return loss_grad(ctx, m, X, y, n, loss);
}

extern "C" lh_status lh_model_adam_step(lh_ctx *ctx, lh_model *m, float lr, float b1, float b2, float eps) {
    if (!ctx || !m) return LH_EINVAL;
    return adam(ctx, m, lr, b1, b2, eps);
}

extern "C" lh_status lh_model_train(lh_ctx *ctx, lh_model *m, const float *X, const float *y, uint32_t n,
                                    uint32_t epochs, uint32_t batch, float lr, uint64_t seed, float *final_loss) {
    if (!ctx || !m || !X || !y || n == 0 || batch == 0) return lh_fail(ctx, LH_EINVAL, "bad argument");
    batch = std::min(batch, n);
    uint32_t *didx = nullptr;
    float *bX = nullptr, *by = nullptr;
    lh_status s = lh_alloc(ctx, &didx, n);
    if (s == LH_OK) s = lh_alloc(ctx, &bX, (size_t)batch * m->n_in);
    if (s == LH_OK) s = lh_alloc(ctx, &by, batch);
    std::vector<uint32_t> perm(n);
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    std::mt19937_64 rng(seed);
    for (uint32_t ep = 0; ep < epochs && s == LH_OK; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        cudaMemcpyAsync(didx, perm.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream);
        for (uint32_t b0 = 0; b0 + batch <= n && s == LH_OK; b0 += batch) {
            LH_TRACED(ctx, "k_gather_rows", k_gather_rows<<<blocks_for((uint64_t)batch * m->n_in), 256, 0, ctx->stream>>>(
                                                X, y, didx + b0, batch, m->n_in, bX, by));
            s = loss_grad(ctx, m, bX, by, batch, m->loss);
            if (s == LH_OK) s = adam(ctx, m, lr, 0.9f, 0.999f, 1e-8f);
        }
        // the host copy of perm is rewritten next epoch: wait for the upload
        if (s == LH_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "train sync");
    }
    if (s == LH_OK && final_loss) {
        s = loss_grad(ctx, m, X, y, n, m->loss);
        if (s == LH_OK) s = lh_readback(ctx, m->loss, sizeof(float), final_loss);
    }
    lh_free(ctx, didx);
    lh_free(ctx, bX);
    lh_free(ctx, by);
    return s;
}

extern "C" lh_status lh_plan_features(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan, lh_trie *const *tries,
                                      float *feat) {
    if (!ctx || !q || !plan || !feat || !tries) return lh_fail(ctx, LH_EINVAL, "null argument");
    lh_trie *et[LH_MAX_EDGES];
    for (uint32_t e = 0; e < q->n_edges; ++e) et[e] = q->edges[e].trie_slot >= 0 ? tries[q->edges[e].trie_slot] : nullptr;
    return features(ctx, q, plan->order, plan->bs_ratio, plan->bs_ratio_inner, et, feat);
}

extern "C" lh_status lh_plan_time(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan, lh_trie *const *tries,
                                  float budget_ms, uint32_t repeats, float *ms) {
    if (!ctx || !q || !plan || !tries || !ms) return lh_fail(ctx, LH_EINVAL, "null argument");
    cudaEvent_t e0, e1;
    LH_CU(cudaEventCreate(&e0));
    LH_CU(cudaEventCreate(&e1));
    lh_status s = LH_OK;
    double tot = 0;
    const uint32_t reps = std::max<uint32_t>(1, repeats);
    for (uint32_t r = 0; r <= reps && s == LH_OK; ++r) {  // run 0 warms up
        lh_result *res = nullptr;
        cudaEventRecord(e0, ctx->stream);
        s = lh_join_dispatch(ctx, q, plan, tries, &res, budget_ms > 0 ? budget_ms : 0.0);
        cudaEventRecord(e1, ctx->stream);
        if (s != LH_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) s = lh_fail(ctx, LH_ECUDA, "plan timing sync");
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        lh_result_free(ctx, res);
        if (r > 0) tot += t;
        if (budget_ms > 0 && t > budget_ms) s = lh_fail(ctx, LH_ETIMEOUT, "plan ran %.1f ms > %.1f ms budget", t, budget_ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == LH_OK) *ms = (float)(tot / reps);
    return s;
}
