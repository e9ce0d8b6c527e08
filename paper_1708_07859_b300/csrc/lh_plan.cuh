// Planner internals shared between the cost model and the learned /
// exhaustive planners.
#pragma once
#include <vector>

#include "lh_internal.cuh"

uint32_t lh_exec_for(const lh_query *q, const uint32_t *order);
int lh_icost_vertex(const lh_query *q, const uint32_t *order, uint32_t i);
void lh_weights(const lh_query *q, const uint64_t *cards, int64_t *w);
int64_t lh_cost_of(const lh_query *q, const uint32_t *order, const int64_t *w);
void lh_candidate_orders(const lh_query *q, std::vector<std::vector<uint32_t>> &out);
lh_status lh_plan_cost(lh_ctx *ctx, const lh_query *q, const uint64_t *cards, lh_plan_t *out);
lh_status lh_plan_learned(lh_ctx *ctx, const lh_query *q, const lh_model *model,
                          const lh_relation_desc *const *rels, const lh_plan_opts *o,
                          const uint64_t *cards, lh_plan_t *out);
lh_status lh_plan_exhaustive(lh_ctx *ctx, const lh_query *q, const lh_relation_desc *const *rels,
                             const lh_plan_opts *o, lh_plan_t *out);
