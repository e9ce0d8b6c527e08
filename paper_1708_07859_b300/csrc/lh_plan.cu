// Planner: the cost-based optimizer of Section 4 (icost x weight over the
// attribute order), the learned alternative (MLP scores over trie features)
// and the exhaustive judge (time every candidate).
#include <chrono>
#include <cmath>
#include <functional>

#include "lh_join.cuh"
#include "lh_plan.cuh"

namespace {

enum Layout { BS = 0, UINT = 1 };

int icost_pair(int a, int b) {
    if (a == BS && b == BS) return 1;
    if (a == UINT && b == UINT) return 50;
    return 10;
}

}  // namespace

// icost of vertex order[i] (Section 4.1.1): relations containing it guess bs
// if none of their vertices came earlier (first trie level), uint otherwise;
// bs sets are intersected first, bs cap uint yields uint; one set (or a
// completely dense relation) needs no intersection.
int lh_icost_vertex(const lh_query *q, const uint32_t *order, uint32_t i) {
    const uint32_t v = order[i];
    int layouts[LH_MAX_EDGES];
    int n = 0;
    for (uint32_t e = 0; e < q->n_edges; ++e) {
        const lh_edge &E = q->edges[e];
        if (E.trie_slot < 0) continue;  // completely dense: icost 0
        bool has = false, earlier = false;
        for (uint32_t c = 0; c < E.nattrs; ++c) {
            if (E.attrs[c] == v) has = true;
            for (uint32_t k = 0; k < i; ++k)
                if (E.attrs[c] == order[k]) earlier = true;
        }
        if (has) layouts[n++] = earlier ? UINT : BS;
    }
    if (n <= 1) return 0;
    std::sort(layouts, layouts + n);  // bs first
    int cur = layouts[0], cost = 0;
    for (int k = 1; k < n; ++k) {
        cost += icost_pair(cur, layouts[k]);
        cur = (cur == BS && layouts[k] == BS) ? BS : UINT;
    }
    return cost;
}

// Section 4.2: score = ceil(|r| / |r_heavy| * 100); a vertex weighs the
// highest score among its relations under an equality selection, the lowest
// otherwise.
void lh_weights(const lh_query *q, const uint64_t *cards, int64_t *w) {
    uint64_t heavy = 1;
    for (uint32_t e = 0; e < q->n_edges; ++e) heavy = std::max<uint64_t>(heavy, cards[e]);
    int64_t score[LH_MAX_EDGES];
    for (uint32_t e = 0; e < q->n_edges; ++e) {
        unsigned __int128 num = (unsigned __int128)cards[e] * 100u;
        score[e] = (int64_t)((num + heavy - 1) / heavy);
    }
    for (uint32_t v = 0; v < q->n_attrs; ++v) {
        const bool eq = (q->eq_selected_mask >> v) & 1u;
        int64_t best = eq ? INT64_MIN : INT64_MAX;
        for (uint32_t e = 0; e < q->n_edges; ++e) {
            bool has = false;
            for (uint32_t c = 0; c < q->edges[e].nattrs; ++c) has |= q->edges[e].attrs[c] == v;
            if (!has) continue;
            best = eq ? std::max(best, score[e]) : std::min(best, score[e]);
        }
        w[v] = (best == INT64_MIN || best == INT64_MAX) ? 0 : best;
    }
}

int64_t lh_cost_of(const lh_query *q, const uint32_t *order, const int64_t *w) {
    int64_t c = 0;
    for (uint32_t i = 0; i < q->n_attrs; ++i) c += (int64_t)lh_icost_vertex(q, order, i) * w[order[i]];
    return c;
}

static int icost_sum(const lh_query *q, const uint32_t *order) {
    int s = 0;
    for (uint32_t i = 0; i < q->n_attrs; ++i) s += lh_icost_vertex(q, order, i);
    return s;
}

// Orders with materialized attributes first (Section 4), plus the Section
// 4.1.2 relaxation: swap the last two attributes when the last is projected
// away, the one before it is materialized and the swap lowers the summed icost.
void lh_candidate_orders(const lh_query *q, std::vector<std::vector<uint32_t>> &out) {
    std::vector<uint32_t> mat, proj;
    for (uint32_t v = 0; v < q->n_attrs; ++v)
        ((q->materialized_mask >> v) & 1u ? mat : proj).push_back(v);
    std::sort(mat.begin(), mat.end());
    do {
        std::vector<uint32_t> pp = proj;
        std::sort(pp.begin(), pp.end());
        do {
            std::vector<uint32_t> o = mat;
            o.insert(o.end(), pp.begin(), pp.end());
            out.push_back(o);
            const size_t n = o.size();
            if (n >= 2 && !((q->materialized_mask >> o[n - 1]) & 1u) && ((q->materialized_mask >> o[n - 2]) & 1u)) {
                std::vector<uint32_t> sw = o;
                std::swap(sw[n - 1], sw[n - 2]);
                if (icost_sum(q, sw.data()) < icost_sum(q, o.data())) out.push_back(sw);
            }
        } while (std::next_permutation(pp.begin(), pp.end()));
    } while (std::next_permutation(mat.begin(), mat.end()));
}

uint32_t lh_exec_for(const lh_query *q, const uint32_t *order) {
    // mirrors the pattern checks of the join dispatcher
    if (q->exec != LH_EXEC_AUTO) return q->exec;
    if (q->n_edges == 2 && q->n_group == 1 && q->group[0].anno < 0 && q->n_attrs == 2) {
        const lh_edge *A = nullptr, *X = nullptr;
        for (uint32_t e = 0; e < 2; ++e) (q->edges[e].trie_slot < 0 ? X : A) = &q->edges[e];
        if (A && X && A->nattrs == 2 && order[0] == q->group[0].attr && order[1] == X->attrs[0]) return LH_EXEC_SPMV;
    }
    if (q->n_edges == 2 && q->n_group == 2 && q->n_attrs == 3 && q->edges[0].trie_slot >= 0 && q->edges[1].trie_slot >= 0) {
        const lh_edge &A = q->edges[0], &B = q->edges[1];
        if (A.nattrs == 2 && B.nattrs == 2 && B.attrs[0] == A.attrs[1] && order[0] == A.attrs[0] &&
            order[1] == A.attrs[1] && order[2] == B.attrs[1])
            return LH_EXEC_SPGEMM;
    }
    return LH_EXEC_GENERIC;
}

lh_status lh_plan_cost(lh_ctx *ctx, const lh_query *q, const uint64_t *cards, lh_plan_t *out) {
    int64_t w[LH_MAX_ATTRS] = {0};
    lh_weights(q, cards, w);
    std::vector<std::vector<uint32_t>> cands;
    lh_candidate_orders(q, cands);
    int64_t best = INT64_MAX;
    std::vector<uint32_t> bo;
    for (auto &o : cands) {
        int64_t c = lh_cost_of(q, o.data(), w);
        if (c < best || (c == best && o < bo)) {
            best = c;
            bo = o;
        }
    }
    out->n_attrs = q->n_attrs;
    for (uint32_t i = 0; i < q->n_attrs; ++i) out->order[i] = bo[i];
    out->cost = best;
    out->bs_ratio = 32;
    out->bs_ratio_inner = 32;
    out->exec = lh_exec_for(q, out->order);
    out->predicted_log_ms = NAN;
    out->measured_ms = NAN;
    out->n_candidates = (uint32_t)cands.size();
    (void)ctx;
    return LH_OK;
}

static lh_status edge_cards(lh_ctx *ctx, const lh_query *q, const lh_relation_desc *const *rels, uint64_t *cards) {
    for (uint32_t e = 0; e < q->n_edges; ++e) {
        const lh_edge &E = q->edges[e];
        uint64_t c = E.card;
        if (c == 0 && E.trie_slot < 0) c = E.flat_n;
        if (c == 0 && rels && rels[e]) c = rels[e]->nrows;
        if (c == 0) return lh_fail(ctx, LH_EINVAL, "edge %u: cardinality unknown (set card or pass rels)", e);
        cards[e] = c;
    }
    return LH_OK;
}

extern "C" lh_status lh_plan_explain(lh_ctx *ctx, const lh_query *q, const uint32_t *order, int32_t *icost,
                                     int64_t *weight, int64_t *cost) {
    if (!ctx || !q || !order) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (q->n_attrs == 0 || q->n_attrs > LH_MAX_ATTRS || q->n_edges == 0 || q->n_edges > LH_MAX_EDGES)
        return lh_fail(ctx, LH_EINVAL, "bad query sizes");
    uint32_t seen = 0;
    for (uint32_t i = 0; i < q->n_attrs; ++i) {
        if (order[i] >= q->n_attrs || ((seen >> order[i]) & 1u)) return lh_fail(ctx, LH_EINVAL, "order is not a permutation");
        seen |= 1u << order[i];
    }
    for (uint32_t e = 0; e < q->n_edges; ++e)
        for (uint32_t c = 0; c < q->edges[e].nattrs; ++c)
            if (q->edges[e].attrs[c] >= q->n_attrs) return lh_fail(ctx, LH_EINVAL, "edge %u: attribute out of range", e);
    uint64_t cards[LH_MAX_EDGES];
    LH_TRY(edge_cards(ctx, q, nullptr, cards));
    int64_t w[LH_MAX_ATTRS] = {0};
    lh_weights(q, cards, w);
    for (uint32_t i = 0; i < q->n_attrs; ++i) {
        if (icost) icost[i] = lh_icost_vertex(q, order, i);
        if (weight) weight[i] = w[i];
    }
    if (cost) *cost = lh_cost_of(q, order, w);
    return LH_OK;
}

extern "C" lh_status lh_plan(lh_ctx *ctx, const lh_query *q, lh_planner_kind kind, const lh_model *model,
                             const lh_relation_desc *const *rels, const lh_plan_opts *opts, lh_plan_t *out) {
    if (!ctx || !q || !out) return lh_fail(ctx, LH_EINVAL, "null argument");
    if (q->n_attrs == 0 || q->n_attrs > LH_MAX_ATTRS || q->n_edges == 0 || q->n_edges > LH_MAX_EDGES)
        return lh_fail(ctx, LH_EINVAL, "bad query sizes");
    for (uint32_t e = 0; e < q->n_edges; ++e)
        for (uint32_t c = 0; c < q->edges[e].nattrs; ++c)
            if (q->edges[e].attrs[c] >= q->n_attrs) return lh_fail(ctx, LH_EINVAL, "edge %u: attribute out of range", e);
    memset(out, 0, sizeof(*out));
    uint64_t cards[LH_MAX_EDGES];
    LH_TRY(edge_cards(ctx, q, rels, cards));
    LH_TRY(lh_plan_cost(ctx, q, cards, out));
    if (kind == LH_PLANNER_COST) return LH_OK;
    if (!rels) return lh_fail(ctx, LH_EINVAL, "learned and exhaustive planners need the relations");
    lh_plan_opts o = opts ? *opts : lh_plan_opts{4, {0, 8, 32, 128}, 0.f, 1, 0};
    if (o.n_policies == 0 || o.n_policies > 4) return lh_fail(ctx, LH_EINVAL, "1..4 layout policies");
    if (kind == LH_PLANNER_LEARNED) {
        if (!model) return lh_fail(ctx, LH_EINVAL, "learned planner needs a model");
        return lh_plan_learned(ctx, q, model, rels, &o, cards, out);
    }
    if (kind == LH_PLANNER_EXHAUSTIVE) return lh_plan_exhaustive(ctx, q, rels, &o, out);
    return lh_fail(ctx, LH_EINVAL, "unknown planner kind");
}
