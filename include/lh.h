/*
 * lh.h -- C ABI of the B300 (sm_103a) worst-case-optimal join-aggregate
 * engine, the hot path of LevelHeaded (arXiv 1708.07859).
 *
 * Conventions for every entry point
 *   - Returns lh_status; no exception or abort crosses the ABI.  On failure
 *     lh_last_error(ctx) holds a one-line reason.
 *   - "device" pointers are CUDA global-memory addresses on the context's
 *     device; "host" pointers are ordinary host memory.  Host structs are
 *     copied during the call.  Device inputs are caller-owned and must stay
 *     valid until the work that reads them is complete (lh_sync /
 *     lh_result_wait).
 *   - All work is issued asynchronously on the context's CUDA stream.  Calls
 *     that size an allocation from device data read a few words back and so
 *     synchronise the stream there: lh_build_trie (level sizes and bitset
 *     totals, plus the key maxima when no key_bound is given), the SpGEMM
 *     path of lh_join_aggregate (the product bound), and the generic join
 *     driver (frontier sizes between chunks).  Device-side error words
 *     (overflow, bounded-wait timeouts) surface at the call's own readback,
 *     at lh_sync or at lh_result_wait.
 *   - Objects returned through out-pointers (tries, results, models,
 *     batches) own device memory until their *_free call.
 */
#ifndef LH_H
#define LH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LH_MAX_LEVELS 6  /* key attributes of one relation (trie levels) */
#define LH_MAX_ATTRS 6   /* key attributes of one query (hypergraph vertices) */
#define LH_MAX_EDGES 8   /* relations of one query (hyperedges) */
#define LH_MAX_ANNOS 4   /* annotation columns of one relation */
#define LH_NFEAT 64      /* learned-planner feature vector length */
#define LH_MAX_GROUP 6   /* GROUP BY columns of one query */

typedef enum {
    LH_OK = 0,
    LH_EINVAL = 1,        /* bad argument */
    LH_ENOMEM = 2,        /* device allocation failed */
    LH_ECUDA = 3,         /* CUDA runtime error */
    LH_ETIMEOUT = 4,      /* a bounded device wait or a host time budget ran out */
    LH_EUNSUPPORTED = 5,  /* shape outside what this build handles */
    LH_EOVERFLOW = 6      /* a 32-bit offset or capacity would overflow */
} lh_status;

/* Commutative semirings of the aggregation (AJAR, Section 2.3). */
typedef enum {
    LH_COUNT_U64 = 0,      /* (N, +, x), every tuple annotated 1 */
    LH_SUM_F32_KAHAN = 1,  /* sum of the product of annotations, fp32 compensated,
                              fp64 final per-group totals */
    LH_SUM_F64 = 2,        /* as above, totals reported in fp64 (same kernels) */
    LH_SUMPROD_F32 = 3     /* sum-product of fp32 annotations (sparse LA) */
} lh_semiring;

typedef enum { LH_T_F32 = 0, LH_T_F64 = 1, LH_T_I8 = 2, LH_T_I32 = 3, LH_T_U32 = 4 } lh_dtype;

typedef struct lh_ctx lh_ctx;
typedef struct lh_trie lh_trie;
typedef struct lh_result lh_result;
typedef struct lh_model lh_model;
typedef struct lh_batch lh_batch;

/* ------------------------------------------------------------------ context */

/* Create a context on the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = legacy default stream) on which all work is issued.  Device memory
 * comes from a private stream-ordered memory pool of the context (allocated
 * and freed on that stream); the pool keeps freed memory for reuse until
 * lh_destroy. */
lh_status lh_create(lh_ctx **out, void *cuda_stream);

/* Device memory from the caller's allocator instead of the context's pool
 * (for an application whose framework owns the GPU's memory, e.g. a
 * caching allocator).  alloc returns `bytes` of device memory usable by work
 * issued on `cuda_stream` after the call (NULL on failure: the library call
 * then returns LH_ENOMEM); free releases a pointer the library no longer
 * needs, possibly while work that reads it is still queued on the stream, so
 * the memory may only be reused by work ordered after that (the semantics of
 * a stream-ordered or single-stream caching allocator).  user is passed
 * through unchanged. */
typedef struct {
    void *(*alloc)(uint64_t bytes, void *cuda_stream, void *user);
    void (*free)(void *ptr, void *cuda_stream, void *user);
    void *user;
} lh_alloc_fns;

/* lh_create with the caller's allocator for every device allocation of the
 * context (fns copied; alloc and free must be non-NULL).  lh_pool_reserve
 * and lh_pool_usage then return LH_EUNSUPPORTED. */
lh_status lh_create_with_allocator(lh_ctx **out, void *cuda_stream, const lh_alloc_fns *fns);
lh_status lh_destroy(lh_ctx *ctx);
lh_status lh_set_stream(lh_ctx *ctx, void *cuda_stream);
/* Maps `bytes` of device memory into the context's pool up front (one
 * allocation, freed at once and kept), so that later temporaries of varying
 * sizes are carved from one mapping instead of growing the pool call by
 * call.  Blocks until done; LH_ENOMEM if the device cannot provide it. */
lh_status lh_pool_reserve(lh_ctx *ctx, uint64_t bytes);
/* Bytes of the context's pool handed out right now (used_now) and the most
 * ever handed out at once since the last reset (used_high); either pointer
 * may be NULL.  reset_high != 0 then restarts the high-water mark at the
 * current use.  Read on the host without waiting for the stream: call
 * lh_sync first to see the work issued so far.  No paper counterpart; a
 * diagnostic of this library's memory management. */
lh_status lh_pool_usage(lh_ctx *ctx, uint64_t *used_now, uint64_t *used_high, int reset_high);
/* Last error message of this context (never NULL). */
const char *lh_last_error(const lh_ctx *ctx);
/* Wait for the stream; return the first device-side error word, if any. */
lh_status lh_sync(lh_ctx *ctx);
/* Diagnostic of the bounded device waits (no paper counterpart): launches
 * one warp that waits, at most `spins` tries (1 .. 2^20), on an mbarrier
 * nothing arrives at, then waits for the stream.  Returns LH_ETIMEOUT, the
 * status every mbarrier / TMA wait of this library reports when a copy never
 * completes; the context stays usable afterwards.  LH_EINVAL for bad spins. */
lh_status lh_selftest_bounded_wait(lh_ctx *ctx, uint32_t spins);
/* Library version string. */
const char *lh_version(void);
/* Blocking copies between a device pointer and host memory on the context
 * stream (for reading result arrays back); bytes may be 0. */
lh_status lh_copy_d2h(lh_ctx *ctx, void *host, const void *dev, uint64_t bytes);
lh_status lh_copy_h2d(lh_ctx *ctx, void *dev, const void *host, uint64_t bytes);

/* Kernel tracing.  While enabled, every kernel this context launches is
 * bracketed by two CUDA events recorded on the context stream (the stream it
 * is launched on).  lh_trace_read waits for the stream and reports, per
 * kernel name, the number of launches and the summed event time since the
 * last lh_trace_reset; *n receives the number of names (entries beyond cap
 * are not written). */
typedef struct {
    char name[40];
    uint64_t launches;
    double total_ms;
} lh_trace_entry;
lh_status lh_trace_enable(lh_ctx *ctx, int on);
/* Restricts the events to kernels named `name` (NULL or "" = every kernel);
 * the other kernels are still counted in launches, with total_ms 0. */
lh_status lh_trace_only(lh_ctx *ctx, const char *name);
lh_status lh_trace_read(lh_ctx *ctx, lh_trace_entry *out, uint32_t cap, uint32_t *n);
lh_status lh_trace_reset(lh_ctx *ctx);

/* ------------------------------------------------------ tries (Section 2.2) */

/* A relation as key columns and annotation columns (Section 2.1: keys join,
 * annotations aggregate).  All column pointers are device pointers of length
 * nrows.  Keys are dictionary-encoded uint32 (identity encoding). */
typedef struct {
    uint64_t nrows;
    uint32_t nkeys;
    const uint32_t *keys[LH_MAX_LEVELS];
    uint32_t nannos;
    const void *annos[LH_MAX_ANNOS];
    uint32_t anno_types[LH_MAX_ANNOS]; /* lh_dtype */
    /* Optional domain size of each key column: every value is < key_bound[c]
     * (a matrix's dimensions, a dimension table's cardinality); 0 = unknown.
     * When every key column has one, the build takes its bit widths from
     * them instead of reading the columns' maxima back. */
    uint32_t key_bound[LH_MAX_LEVELS];
} lh_relation_desc;

/* How annotations of duplicate key tuples merge (every tuple has one
 * annotation, Section 2.3), and which annotation the trie stores.
 *   LH_MERGE_SUM: float columns (f32/f64) are summed per distinct tuple.
 *   LH_MERGE_FIRST: the annotation of the first row of the run is kept
 *     (dimension attributes reached through the metadata container M).
 *   LH_MERGE_PRICE_DISCOUNT: annos[0] = price (f64 or f32), annos[1] =
 *     discount in hundredths (i8); the stored annotation is the expression
 *     price * (1 - discount/100) (Section 3.1, rule 3) as an fp32 compensated
 *     pair (two f32 columns: high part, low part), duplicates summed. */
typedef enum { LH_MERGE_SUM = 0, LH_MERGE_FIRST = 1, LH_MERGE_PRICE_DISCOUNT = 2 } lh_merge;

/* Per-set layout choice (Section 2.2: dense sets as bitsets, sparse sets as
 * sorted uint32).  A set of cardinality c spanning s = max - min + 1 values
 * gets a bitset when its level's ratio r > 0, c >= bs_min_card and c * r >=
 * s.  r is bs_ratio for every level, or level_ratio[l] for level l when
 * per_level != 0 (a policy per trie level).  NULL selects {32, 32}.  Every
 * set keeps its sorted uint32 array (used to iterate); a bitset set
 * additionally has 32-bit words (base = min rounded down to 128, word count
 * a multiple of 4) and a per-word rank. */
typedef struct {
    uint32_t bs_ratio;
    uint32_t bs_min_card;
    uint32_t per_level;
    uint32_t level_ratio[LH_MAX_LEVELS];
} lh_layout_policy;

/* Build the trie of `rel` with level l holding key column key_order[l]
 * (key_order: host array, a permutation of [0, nkeys)).  Radix-sorts the
 * packed key tuples (total key bits <= 64), removes duplicates merging their
 * annotations per `merge`, emits CSR levels, decides each set's layout and
 * gathers annotations into leaf order.  Synchronises to size the levels and
 * the bitset arena, and once more to read the key maxima unless every key
 * column has a key_bound.  Errors: LH_EINVAL (bad order, nkeys 0 or >
 * LH_MAX_LEVELS, merge/type mismatch, a key value at or above its declared
 * key_bound), LH_EUNSUPPORTED (> 64 packed key bits), LH_EOVERFLOW (a level
 * larger than 2^32 - 1 entries), LH_ETIMEOUT (a bounded device wait gave up),
 * LH_ENOMEM. */
lh_status lh_build_trie(lh_ctx *ctx, const lh_relation_desc *rel, const uint32_t *key_order,
                        const lh_layout_policy *layout, lh_merge merge, lh_trie **out);

/* Selection pushed into its own relation (Section 3.2): a one-level trie of
 * the keys k in [0, n) with lo <= col[k] <= hi (col: device int32, length n).
 * Its single set gets the bitset layout whenever the policy allows. */
lh_status lh_filter_trie(lh_ctx *ctx, const int32_t *col, uint64_t n, int32_t lo, int32_t hi,
                         const lh_layout_policy *layout, lh_trie **out);

/* A selection on a relation's rows: keep row r when lo <= col[r] <= hi
 * (col: device int32, one value per row -- a key or an annotation of the
 * relation, e.g. a date or a dictionary-encoded name). */
typedef struct {
    const int32_t *col;
    int32_t lo, hi;
} lh_row_filter;

/* lh_build_trie over only the rows of `rel` that pass every filter of
 * where[0 .. n_where) (0..4): the selection pushed below the joins into a
 * GHD node of its own (Section 3.2), whose relation is the selected one.
 * Compacts the passing rows (one readback of their count), then builds as
 * lh_build_trie does.  Errors as lh_build_trie, plus LH_EINVAL for more than
 * four filters or a null filter column. */
lh_status lh_build_trie_where(lh_ctx *ctx, const lh_relation_desc *rel, const uint32_t *key_order,
                              const lh_layout_policy *layout, lh_merge merge, const lh_row_filter *where,
                              uint32_t n_where, lh_trie **out);

lh_status lh_trie_free(lh_ctx *ctx, lh_trie *t);

typedef struct {
    uint32_t nlevels;
    uint32_t key_order[LH_MAX_LEVELS];
    uint64_t nrows_in;                     /* rows before duplicate removal */
    uint64_t level_n[LH_MAX_LEVELS];       /* entries per level */
    uint64_t level_sets[LH_MAX_LEVELS];    /* sets per level */
    uint64_t level_bs_sets[LH_MAX_LEVELS]; /* of which bitset layout */
    uint64_t bitset_words;
    uint64_t device_bytes;
} lh_trie_stats;

lh_status lh_trie_stats_get(lh_ctx *ctx, const lh_trie *t, lh_trie_stats *out);

/* Device view of one level.  Sets of level l are indexed by their parent
 * entry in level l-1 (level 0 has one set, index 0).  The children of entry
 * p are vals_{l+1}[child_offs[p] .. child_offs[p+1]).  bs_slot[set] is the
 * set's bitset slot or 0xFFFFFFFF; bs_meta[4*slot + {0,1,2,3}] = {first
 * word, base value, word count, rank base}; rank[w] = set bits of the whole
 * bitset arena before word w, so the index of value v in its set is
 * rank[w] - rank base + popc(word w below v's bit). */
typedef struct {
    uint64_t n;
    uint64_t nsets;
    const uint32_t *vals;
    const uint32_t *child_offs; /* NULL at the leaf level */
    const uint32_t *bs_slot;    /* NULL when the level has no bitset set */
    uint64_t n_bs;
    const uint32_t *bs_meta;
    const uint32_t *words;
    const uint32_t *rank;
} lh_level_view;

lh_status lh_trie_level(lh_ctx *ctx, const lh_trie *t, uint32_t level, lh_level_view *out);
/* Annotation column `col` in leaf order (device pointer) and its lh_dtype. */
lh_status lh_trie_anno(lh_ctx *ctx, const lh_trie *t, uint32_t col, const void **ptr,
                       uint32_t *dtype);

/* ------------------------------------- set intersection (Section 4.1.1, Fig 4a) */

/* One set: layout 0 = sorted distinct uint32 (n elements at data), layout 1 =
 * bitset (n 32-bit words at data, bit b of word w is value base + 32 w + b;
 * base a multiple of 128, data 16-byte aligned, n a multiple of 4). */
typedef struct {
    uint32_t layout;
    uint32_t base;
    uint64_t n;
    const uint32_t *data;
} lh_set;

/* counts[p] = |A[p] cap B[p]| for p < npairs.  a, b, counts: device arrays.
 * uint cap uint uses a merge-path partition of each pair across CTAs when
 * the sizes are within 32x of each other and a binary-search probe of the
 * smaller into the larger otherwise; uint cap bs tests bits; bs cap bs ANDs
 * 128-bit words.  Count-only (Section 2.4: the core operation of an
 * attribute).  Merge tiles and the other kinds run in two kernels (at most
 * two launches); the tile count is read back once, so the call
 * synchronises the context stream there. */
lh_status lh_intersect_count_batch(lh_ctx *ctx, uint32_t npairs, const lh_set *a,
                                   const lh_set *b, uint64_t *counts);

/* Same result as lh_intersect_count_batch, for callers that cannot allocate
 * device memory while they run queries -- for instance a host application
 * whose buffer pool or framework allocator owns all of the GPU's memory, or
 * a latency-bound loop where an allocation could stall or fail.  The paper
 * has no counterpart; this is a property of this library's interface.
 *   - Allocates nothing: no cudaMalloc/cudaFree, no stream-ordered pool.
 *     Its scratch (about 40 bytes per pair) lives in one fixed device array
 *     sized for 65536 pairs (about 2.6 MB) that every GPU loading this
 *     library holds until the process exits.
 *   - npairs above 65536 is rejected with LH_EINVAL (counts untouched).
 *   - The first call on a device looks the array's address up with that
 *     device current (the context's device must be the current device);
 *     make that first call before any stream capture.
 *   - All calls share the array: calls whose work overlaps on the GPU (on
 *     different streams, or from different contexts on one device) race and
 *     give wrong counts; serialise them.
 * a, b, counts: device arrays as for lh_intersect_count_batch; counts is
 * zeroed, then written. */
lh_status lh_intersect_count_batch_noalloc(lh_ctx *ctx, uint32_t npairs, const lh_set *a,
                                           const lh_set *b, uint64_t *counts);

/* ----------------------------------------------- queries (Sections 2.3, 3.1) */

/* A hyperedge: relation `trie_slot` of the tries[] argument whose raw key
 * column c is query attribute attrs[c].  trie_slot = -1 marks a completely
 * dense unary relation over attrs[0] (a flat fp32 buffer `flat` of length
 * flat_n: key k present iff k < flat_n, annotation flat[k]); it needs no
 * intersection (Section 4.1.1, icost 0).  anno: annotation column of the
 * trie multiplied into each result tuple (-1 = identity).  card: relation
 * cardinality for the planner (0 = read it from the trie). */
typedef struct {
    int32_t trie_slot;
    uint32_t nattrs;
    uint32_t attrs[LH_MAX_LEVELS];
    int32_t anno;
    const float *flat;
    uint64_t flat_n;
    uint64_t card;
} lh_edge;

/* A GROUP BY column: the int32 annotation column `anno` of edge `edge`'s trie
 * read at the edge's leaf position (a dimension attribute, Section 5 GROUP BY
 * annotation), or, with anno = -1, the value of key attribute `attr`.
 * card > 0 declares the domain: values must lie in [0, card) (a value
 * outside it is reported as LH_EINVAL at the wait).  card = 0: the domain is
 * unknown, any uint32 value; the query then groups through a hash table. */
typedef struct {
    uint32_t edge;
    int32_t anno;
    uint32_t attr;
    uint32_t card;
} lh_group;

typedef enum {
    LH_EXEC_AUTO = 0,
    LH_EXEC_GENERIC = 1, /* attribute-at-a-time frontier expansion (Algorithm 1) */
    LH_EXEC_SPMV = 2,    /* A(i,j) x(j) group by i, x completely dense */
    LH_EXEC_SPGEMM = 3   /* A(i,j) B(j,k) group by (i,k), j projected away */
} lh_exec;

typedef struct {
    uint32_t n_attrs;
    uint32_t n_edges;
    lh_edge edges[LH_MAX_EDGES];
    uint32_t semiring;          /* lh_semiring */
    uint32_t n_group;           /* 0..LH_MAX_GROUP */
    lh_group group[LH_MAX_GROUP];
    uint32_t materialized_mask; /* bit a: attribute a is an output (materialized) */
    uint32_t eq_selected_mask;  /* bit a: an equality selection touches attribute a */
    uint32_t exec;              /* lh_exec hint */
    uint32_t group_impl;        /* lh_group_impl */
    uint64_t group_capacity;    /* hash GROUP BY: slots of the shared table (0 = twice the product of the
                                   columns' domains -- declared cards, else the distinct values their
                                   relations can hold -- clamped to [2^12, 2^24]) */
    uint32_t isect_impl;        /* lh_isect_impl */
} lh_query;

/* How the generic driver intersects at the last attribute of a COUNT query
 * without GROUP BY when that attribute joins exactly two stored relations
 * (Algorithm 1's innermost intersection, of which only the size is used).
 *   LH_ISECT_AUTO: frontier entries whose smaller set holds at least 32
 *     elements are counted by warps in work items of at most 2048 elements
 *     (a hub's pair spreads over many warps): merge path when both sets are
 *     uint and within 8x of each other in size (windows of 32 elements of
 *     each, matches found with shuffles and counted with a ballot); else the
 *     elements of one set are probed in the other (a bitset word, or a
 *     binary search whose lower end advances with the sorted probes).
 *     Smaller entries take the LH_ISECT_PROBE path.
 *   LH_ISECT_PROBE: one thread per element of the smaller set, probed in the
 *     other (the path of every other attribute).
 * Both give the same count. */
typedef enum { LH_ISECT_AUTO = 0, LH_ISECT_PROBE = 1 } lh_isect_impl;

/* How a GROUP BY on annotations (or keys) accumulates (Section 5).
 *   LH_GROUP_AUTO: dense per-group arrays when at most two columns all
 *     declare a card and the domain product is <= 2^26; otherwise the
 *     paper's rule on the key tuple's width: at most three values -> private
 *     tables, more -> the shared table.
 *   LH_GROUP_DENSE: dense arrays (needs declared cards, product <= 2^26).
 *   LH_GROUP_PRIVATE: every warp upserts into its own open-addressing table
 *     in shared memory (the analog of the paper's per-thread hash maps; no
 *     contention between warps); a full table spills into the shared table,
 *     and each block merges its tables into it at the end.  Needs the packed
 *     key (declared cards' bit widths, 32 bits per undeclared column) to fit
 *     in 63 bits.
 *   LH_GROUP_SHARED: one concurrent open-addressing table in device memory
 *     (the analog of the paper's concurrent cuckoo map): slots claimed by
 *     compare-and-swap on a 64-bit tag, the key tuple stored beside it, fp64
 *     sums and uint64 counts added atomically.
 * The hash paths report their groups as key tuples (lh_result_view
 * group_keys); a shared table that fills up reports LH_EOVERFLOW at the
 * wait.
 * Under LH_EXEC_SPGEMM the field picks how each row of C groups its
 * products by output column (Section 5, the bitset + dense array against
 * the hash table of Figure 5a): under AUTO rows of at most 256 products
 * (and 32 entries of A) sort in registers, and a larger row takes a
 * shared-memory bitset and dense fp64 array when its possible columns span
 * at most 4096 values and its product bound fills at least a quarter of that
 * span, else a hash table; DENSE takes the bitset and array for every row
 * whose span fits; PRIVATE and SHARED never do.  The result (CSR, columns
 * ascending) is the same under every choice. */
typedef enum {
    LH_GROUP_AUTO = 0,
    LH_GROUP_DENSE = 1,
    LH_GROUP_PRIVATE = 2,
    LH_GROUP_SHARED = 3
} lh_group_impl;

/* --------------------------------------------------- planner (Section 4) */

typedef enum { LH_PLANNER_COST = 0, LH_PLANNER_LEARNED = 1, LH_PLANNER_EXHAUSTIVE = 2 } lh_planner_kind;

typedef struct {
    uint32_t n_attrs;
    uint32_t order[LH_MAX_ATTRS]; /* attribute order: order[0] is processed first */
    uint32_t bs_ratio;            /* layout policy of the tries this plan runs on (0 = uint only) */
    uint32_t exec;                /* lh_exec actually used */
    int64_t cost;                 /* Section 4 cost estimate of `order` */
    float predicted_log_ms;       /* learned model output (NaN if not used) */
    float measured_ms;            /* exhaustive timing of the chosen plan (NaN if not used) */
    uint32_t n_candidates;        /* plans considered */
    uint32_t bs_ratio_inner;      /* layout ratio of trie levels >= 1 (bs_ratio: level 0) */
} lh_plan_t;

/* Planner options.  time_budget_ms bounds each exhaustive candidate run
 * (host-side: chunks stop being issued once it is exceeded; the candidate is
 * then ranked last).  policies: layout ratios tried (0 = uint only); with
 * per_level != 0 every (level-0 ratio, inner-level ratio) pair of them is a
 * candidate layout, else one ratio serves every level. */
typedef struct {
    uint32_t n_policies;
    uint32_t policies[4];
    float time_budget_ms;
    uint32_t repeats;
    uint32_t per_level;
} lh_plan_opts;

/* Choose an attribute order (and layout policy) for `q`.
 *   LH_PLANNER_COST: Section 4 cost model (icost x weight, materialized
 *     attributes first, Section 4.1.2 relaxation, ties to the
 *     lexicographically smallest order); needs only edge cardinalities.
 *   LH_PLANNER_LEARNED: scores every (order, policy) with `model` on
 *     features of tries built from `rels` (both key orders of each relation).
 *   LH_PLANNER_EXHAUSTIVE: builds the tries of every candidate from `rels`,
 *     runs and times each, keeps the fastest.
 * rels: host array of n_edges relation descriptors (may repeat), needed for
 * LEARNED and EXHAUSTIVE, else NULL.  opts may be NULL. */
lh_status lh_plan(lh_ctx *ctx, const lh_query *q, lh_planner_kind kind, const lh_model *model,
                  const lh_relation_desc *const *rels, const lh_plan_opts *opts, lh_plan_t *out);

/* The Section 4 cost terms of running q in `order` (host array of
 * q->n_attrs attribute ids, a permutation): icost[i] (host, n_attrs
 * entries) of order position i under the layout guesses of Section 4.1.1,
 * weight[a] (host, n_attrs entries) of attribute a per Section 4.2 from the
 * edges' cardinalities, and *cost = sum_i icost[i] * weight[order[i]].  Any
 * output pointer may be NULL.  The same arithmetic LH_PLANNER_COST
 * minimises; no device work.  LH_EINVAL for a bad order or an edge whose
 * cardinality is unknown. */
lh_status lh_plan_explain(lh_ctx *ctx, const lh_query *q, const uint32_t *order, int32_t *icost,
                          int64_t *weight, int64_t *cost);

/* Key order (host array, edge's nattrs entries) of the trie edge `e` must be
 * built with under `plan`: its key columns sorted by position in plan->order. */
lh_status lh_edge_key_order(const lh_query *q, const lh_plan_t *plan, uint32_t e,
                            uint32_t *key_order);

/* -------------------------------------- join-aggregate (Algorithm 1, Sec 5) */

/* Result of one join-aggregate.  Device pointers stay valid until
 * lh_result_free.  GENERIC: count / sum totals and, with GROUP BY, the dense
 * per-group arrays (group g = g0 * card1 + g1).  SPMV: y (fp32, nrows).
 * SPGEMM: CSR C over the nrows distinct rows of A (c_row: their ids,
 * c_off: nrows+1 uint64, c_col uint32 ascending per row, c_val fp32).  The
 * first nnz entries of c_col / c_val hold C; their allocation is the product
 * bound sum_i sum_{k in A_i} |B_k|, so the join needs no readback of nnz. */
typedef struct {
    uint32_t exec;
    uint64_t count;
    double sum;
    uint32_t ngroups;
    const double *group_sum;
    const uint64_t *group_count;
    uint64_t nrows;
    const float *y;
    uint64_t nnz;
    const uint32_t *c_row;      /* SPGEMM: row id of CSR row r (A's distinct rows, ascending) */
    const uint64_t *c_off;
    const uint32_t *c_col;
    const float *c_val;
    uint64_t elements;          /* intersection input elements examined (probe count) */
    /* hash GROUP BY (group_impl PRIVATE / SHARED): ngroups groups in no
     * particular order; group g's key is group_keys[c * ngroups + g] for
     * column c < n_group_cols; group_sum / group_count hold its totals */
    uint32_t n_group_cols;
    const uint32_t *group_keys;
    uint32_t group_impl;        /* lh_group_impl the join used */
    /* generic driver: set elements its intersections read -- every
     * candidate of the smallest (driving) set plus one probe (a bitset word
     * or a searched element) into each other set -- the data a count of
     * `elements` boils down to when the larger sets are probed, not scanned */
    uint64_t visited;
} lh_result_view;

/* Run query q under plan.  tries: host array of device tries, indexed by
 * edge.trie_slot; each edge's trie must have been built with the key order
 * lh_edge_key_order gives for this plan (checked: LH_EINVAL otherwise).
 * COUNT, SUM (compensated fp32, fp64 totals) and GROUP BY on up to
 * LH_MAX_GROUP columns (dense arrays or hash tables, see lh_group_impl) are
 * supported by the generic driver. */
lh_status lh_join_aggregate(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan,
                            lh_trie *const *tries, lh_result **out);
/* The result of q under plan as a relation of its own: one tuple per
 * distinct value combination of the key attributes out_attrs[0 .. n_out)
 * among the join results, annotated with the aggregate of the tuples under
 * it -- the semiring sum of the annotation products (the number of join
 * results for LH_COUNT_U64) -- as a compensated fp32 pair (annotation
 * columns 0 and 1, f32 high and low parts, which a later join multiplies as
 * one annotation).  This is the intermediate result an inner node of a GHD
 * plan hands to its parent (Sections 2.3 and 3.2: the node's output is
 * projected onto the attributes it shares with the parent, the others
 * aggregated away).  The returned trie has levels in out_attrs order.
 * Groups through the hash GROUP BY (group_impl AUTO picks private or shared
 * tables); synchronises.  Errors as lh_join_aggregate and lh_build_trie. */
lh_status lh_join_to_trie(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan, lh_trie *const *tries,
                          uint32_t n_out, const uint32_t *out_attrs, const lh_layout_policy *layout,
                          lh_trie **out);
/* Wait for the result and fill `view` (host struct; device pointers inside;
 * for SPGEMM this is where nnz is read back). */
lh_status lh_result_wait(lh_ctx *ctx, lh_result *r, lh_result_view *view);
lh_status lh_result_free(lh_ctx *ctx, lh_result *r);

/* ------------------------------------------------ dense block (Section 3.1) */

/* C = A B for dense fp32 A (m x k, row-major) and B (k x n, row-major), the
 * flat annotation buffers attribute elimination leaves (Section 3.1).  A and
 * B are split into bf16 high parts and bf16 residuals; the product of the
 * high parts runs on tcgen05 tensor cores with fp32 accumulators in tensor
 * memory and is written to c_bf16 (fp32, m x n); one refinement step adds
 * the two residual cross products (fp32 accumulation) and writes the sum in
 * fp64 to c_refined (m x n; may be NULL to skip the refinement).  m, n, k
 * must be multiples of 128, 256 and 64 respectively (LH_EUNSUPPORTED
 * otherwise).  Scratch: 4 bf16 copies of the inputs, from the stream's pool. */
lh_status lh_dense_matmul(lh_ctx *ctx, const float *A, const float *B, int m, int n, int k,
                          float *c_bf16, double *c_refined);

/* y = A x for a dense fp32 A (m x n, row-major) and x (n): the dense
 * matrix-vector product attribute elimination leaves (Section 3.1: a single
 * dense annotation in a flat, BLAS-compatible buffer; the DMV rows of
 * Section 6.2 / Table 1).  Products are split error-free and summed as
 * compensated fp32 pairs; y (fp32, m) receives the rounded sums and, when
 * y_refined is not NULL, y_refined (fp64, m) the pairs' exact sums.  Any m,
 * n >= 0; rows are read with 16-byte loads when n is a multiple of 4 and A
 * and x are 16-byte aligned.  No scratch memory; asynchronous on the
 * context stream. */
lh_status lh_dense_matvec(lh_ctx *ctx, const float *A, const float *x, int m, int n, float *y,
                          double *y_refined);

/* --------------------------------- batched uneven joins (no paper counterpart) */

typedef enum { LH_BATCH_TRIANGLE = 0, LH_BATCH_CLIQUE4 = 1 } lh_batch_kind;

/* One query of a batch: COUNT of the triangle (or 4-clique) join over the
 * oriented edge relation E held in `graph`, a 2-level trie built with key
 * order {0, 1} from edges (src < dst). */
typedef struct {
    uint32_t kind;
    const lh_trie *graph;
} lh_batch_query;

/* Work-splitting thresholds of the persistent kernel: an outer vertex with
 * at most t_warp out-edges is handled by one warp with the whole edge range;
 * larger ones are split into chunks of `chunk` edges; ctas_per_sm sets the
 * persistent grid (148 SMs x ctas_per_sm CTAs of 256 threads). */
typedef struct {
    uint32_t t_warp;
    uint32_t chunk;
    uint32_t ctas_per_sm;
    uint32_t reserved;
} lh_batch_tuning;

/* Pack n queries into one work list and capture one persistent launch (plus
 * the reset of its counters) in a CUDA graph.  counts: device uint64[n],
 * written by every lh_batch_run.  tuning NULL = defaults. */
lh_status lh_batch_create(lh_ctx *ctx, uint32_t n, const lh_batch_query *qs,
                          const lh_batch_tuning *tuning, uint64_t *counts, lh_batch **out);
/* Replay the captured graph on the context stream. */
lh_status lh_batch_run(lh_ctx *ctx, lh_batch *b);
lh_status lh_batch_free(lh_ctx *ctx, lh_batch *b);
/* Input set elements of the intersections the last replay executed (for
 * each intersection the cardinalities of every set taking part: the
 * throughput measure of the join); waits for the stream. */
lh_status lh_batch_elements(lh_ctx *ctx, lh_batch *b, uint64_t *elements);
/* Sweep tunings (successive halving over a grid of t_warp, chunk and
 * ctas_per_sm) and return the fastest.  The candidates are timed on a fixed
 * sample of the batch -- every 4th query, or all of them when n < 8 -- so the
 * other queries stay out of the tuning.  best_ms: the winner's replay time on
 * that sample.  counts (device uint64[n]) is scratch while tuning. */
lh_status lh_batch_autotune(lh_ctx *ctx, uint32_t n, const lh_batch_query *qs, uint64_t *counts,
                            lh_batch_tuning *best, float *best_ms);

/* The batched form of lh_join_aggregate: n queries with their plans;
 * tries[i] is query i's host array of tries (as for lh_join_aggregate);
 * out: host array of n result handles, each read with lh_result_wait and
 * released with lh_result_free as usual.  Queries the persistent kernel
 * serves -- COUNT without GROUP BY of the triangle R(a,b) S(b,c) T(a,c) or of
 * the six-edge 4-clique over one relation, in the identity attribute order,
 * every edge on the same trie built in key order {0, 1} -- are packed into
 * one graph-captured launch (tuning as for lh_batch_create, NULL =
 * defaults) and are complete when the call returns (one synchronisation for
 * all of them; their result views report count only).  Every other query
 * runs through lh_join_aggregate in turn.  On failure no result is
 * returned (all of out[] is NULL). */
lh_status lh_join_aggregate_batch(lh_ctx *ctx, uint32_t n, const lh_query *qs, const lh_plan_t *plans,
                                  lh_trie *const *const *tries, const lh_batch_tuning *tuning,
                                  lh_result **out);

/* ------------------------------------ learned cost model (no paper counterpart) */

/* MLP n_in -> hidden -> hidden -> 1 with ReLU, fp32, parameters in one flat
 * device buffer: W1 (n_in x hidden, row-major), b1, W2 (hidden x hidden), b2,
 * W3 (hidden), b3.  Trained with mean squared error and Adam by this
 * library's own kernels. */
lh_status lh_model_create(lh_ctx *ctx, uint32_t n_in, uint32_t hidden, uint64_t seed,
                          lh_model **out);
lh_status lh_model_free(lh_ctx *ctx, lh_model *m);
/* Device pointers of the flat parameter and gradient buffers and their length. */
lh_status lh_model_buffers(lh_ctx *ctx, lh_model *m, float **params, float **grads,
                           uint64_t *n_params);
/* out[i] = model(X[i]) for X: device fp32 (n x n_in, row-major). */
lh_status lh_model_forward(lh_ctx *ctx, const lh_model *m, const float *X, uint32_t n, float *out);
/* Loss (device fp32 scalar) and gradients (into the model's grad buffer) of
 * mean((model(X) - y)^2). */
lh_status lh_model_loss_grad(lh_ctx *ctx, lh_model *m, const float *X, const float *y, uint32_t n,
                             float *loss);
/* One Adam step on the model's current gradients (bias-corrected). */
lh_status lh_model_adam_step(lh_ctx *ctx, lh_model *m, float lr, float beta1, float beta2,
                             float eps);
/* Minibatch training: epochs x ceil(n / batch) Adam steps over a seeded
 * shuffle; final_loss: host, full-set loss after training. */
lh_status lh_model_train(lh_ctx *ctx, lh_model *m, const float *X, const float *y, uint32_t n,
                         uint32_t epochs, uint32_t batch, float lr, uint64_t seed,
                         float *final_loss);
/* Engine-measured time of q under plan on `tries` (as for
 * lh_join_aggregate): one warm-up run, then the mean of `repeats` runs
 * timed with CUDA events on the context stream, into *ms (host).  With
 * budget_ms > 0 the generic driver stops issuing chunks once a run exceeds
 * the budget and the call returns LH_ETIMEOUT (the planner's training data
 * and exhaustive judge rank such plans last). */
lh_status lh_plan_time(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan, lh_trie *const *tries,
                       float budget_ms, uint32_t repeats, float *ms);
/* Planner features (host float[LH_NFEAT]) of running q under plan on
 * `tries` (built for that plan), from device-side statistics of the tries'
 * levels: [0, 6) log2(1 + |relation|) per edge; [6, 31) per order position
 * d < 5: log2 set-size median, 90th percentile, maximum, level density, and
 * log2(1 + icost(v_d) x weight(v_d)) of the Section 4 cost model; [31, 56)
 * position x attribute one-hot; [56, 60) one-hot of the level-0 layout
 * ratio and [60, 64) of the inner levels' ratio (0, 8, 32, other). */
lh_status lh_plan_features(lh_ctx *ctx, const lh_query *q, const lh_plan_t *plan,
                           lh_trie *const *tries, float *feat);

#ifdef __cplusplus
}
#endif
#endif /* LH_H */
