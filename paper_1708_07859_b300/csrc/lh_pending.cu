// Entry points whose kernels are not in this build yet: they refuse with
// LH_EUNSUPPORTED.
#include "lh_plan.cuh"

lh_status lh_plan_learned(lh_ctx *ctx, const lh_query *, const lh_model *, const lh_relation_desc *const *,
                          const lh_plan_opts *, const uint64_t *, lh_plan_t *) {
    return lh_fail(ctx, LH_EUNSUPPORTED, "learned planner not built");
}
lh_status lh_plan_exhaustive(lh_ctx *ctx, const lh_query *, const lh_relation_desc *const *,
                             const lh_plan_opts *, lh_plan_t *) {
    return lh_fail(ctx, LH_EUNSUPPORTED, "exhaustive planner not built");
}
extern "C" {
lh_status lh_batch_create(lh_ctx *ctx, uint32_t, const lh_batch_query *, const lh_batch_tuning *, uint64_t *, lh_batch **) {
    return lh_fail(ctx, LH_EUNSUPPORTED, "batch not built");
}
lh_status lh_batch_run(lh_ctx *ctx, lh_batch *) { return lh_fail(ctx, LH_EUNSUPPORTED, "batch not built"); }
lh_status lh_batch_free(lh_ctx *ctx, lh_batch *) { return lh_fail(ctx, LH_EUNSUPPORTED, "batch not built"); }
lh_status lh_batch_autotune(lh_ctx *ctx, uint32_t, const lh_batch_query *, uint64_t *, lh_batch_tuning *, float *) {
    return lh_fail(ctx, LH_EUNSUPPORTED, "batch not built");
}
lh_status lh_model_create(lh_ctx *ctx, uint32_t, uint32_t, uint64_t, lh_model **) { return lh_fail(ctx, LH_EUNSUPPORTED, "model not built"); }
lh_status lh_model_free(lh_ctx *ctx, lh_model *) { return lh_fail(ctx, LH_EUNSUPPORTED, "model not built"); }
lh_status lh_model_buffers(lh_ctx *ctx, lh_model *, float **, float **, uint64_t *) { return lh_fail(ctx, LH_EUNSUPPORTED, "model not built"); }
lh_status lh_model_forward(lh_ctx *ctx, const lh_model *, const float *, uint32_t, float *) { return lh_fail(ctx, LH_EUNSUPPORTED, "model not built"); }
lh_status lh_model_loss_grad(lh_ctx *ctx, lh_model *, const float *, const float *, uint32_t, float *) { return lh_fail(ctx, LH_EUNSUPPORTED, "model not built"); }
lh_status lh_model_adam_step(lh_ctx *ctx, lh_model *, float, float, float, float) { return lh_fail(ctx, LH_EUNSUPPORTED, "model not built"); }
lh_status lh_model_train(lh_ctx *ctx, lh_model *, const float *, const float *, uint32_t, uint32_t, uint32_t, float, uint64_t, float *) { return lh_fail(ctx, LH_EUNSUPPORTED, "model not built"); }
lh_status lh_plan_features(lh_ctx *ctx, const lh_query *, const lh_plan_t *, lh_trie *const *, float *) { return lh_fail(ctx, LH_EUNSUPPORTED, "features not built"); }
}
