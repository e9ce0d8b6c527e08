// Shared declarations of the join-aggregate drivers.
#pragma once
#include "lh_internal.cuh"

struct lh_result {
    uint32_t exec = LH_EXEC_GENERIC;
    uint64_t *d_count = nullptr;   // device counter (COUNT without GROUP BY)
    uint64_t host_count = 0;       // counts the driver resolved on the host
    uint64_t *d_elems = nullptr;   // intersection input elements examined
    uint64_t visited = 0;          // elements the intersections read (candidates + one probe per other set)
    uint32_t ngroups = 0;
    double *d_gsum = nullptr;
    uint64_t *d_gcount = nullptr;
    uint64_t nrows = 0;
    float *y = nullptr;
    uint64_t nnz = 0;
    bool nnz_pending = false;  // SPGEMM: nnz = c_off[nrows], read at lh_result_wait
    const uint32_t *c_row = nullptr;
    uint64_t *c_off = nullptr;
    uint32_t *c_col = nullptr;
    float *c_val = nullptr;
    uint32_t semiring = 0;
    // hash GROUP BY: the shared table (compacted into the group arrays at
    // the wait) and the compacted keys
    uint32_t group_impl = LH_GROUP_DENSE;
    uint32_t n_group_cols = 0;
    bool hash_pending = false;
    unsigned long long *ht_tag = nullptr;
    uint32_t *ht_keys = nullptr;
    double *ht_sum = nullptr;
    unsigned long long *ht_cnt = nullptr;
    uint32_t ht_cap = 0;
    uint32_t *group_keys = nullptr;
    std::vector<void *> allocs;
};

template <class T>
static inline lh_status res_alloc(lh_ctx *ctx, lh_result *r, T **p, size_t count) {
    LH_TRY(lh_alloc(ctx, p, count));
    r->allocs.push_back((void *)*p);
    return LH_OK;
}

// Sparse LA drivers (lh_spla.cu).  a: trie of A with levels (i, j) and one
// f32 annotation; b: trie of B with levels (j, k) and one f32 annotation.
lh_status lh_run_spmv(lh_ctx *ctx, const lh_trie *a, const float *x, uint64_t x_n, uint64_t nrows,
                      lh_result *r);
// dense_mode: 0 never the dense-array GROUP BY key, 1 by the density rule,
// 2 every row whose output span fits it
lh_status lh_run_spgemm(lh_ctx *ctx, const lh_trie *a, const lh_trie *b, lh_result *r, uint32_t dense_mode);

// Generic attribute-at-a-time driver (lh_join.cu).
lh_status lh_run_generic(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan,
                         lh_trie *const *tries, lh_result *r, double deadline_ms);

// Host validation shared by the planner: position of each attribute in the
// plan order, and the key order an edge's trie needs.
bool lh_key_order_for(const lh_query *q, const uint32_t *order, uint32_t n_attrs, uint32_t e,
                      uint32_t *key_order);
