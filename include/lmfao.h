/*
 * lmfao.h -- C ABI of a B300 (sm_103a) engine for batches of group-by aggregates
 * over the natural join of an acyclic schema.
 *
 * The problem (Section 1, Section 2 of "LMFAO: An Engine for Batches of Group-By
 * Aggregates"): given relations R_1..R_m whose attributes with equal names are
 * equated (the natural join D), evaluate many queries of the form
 *
 *     SELECT G, SUM(prod_i f_i(x)), ... FROM D WHERE cond GROUP BY G
 *
 * in one plan, bottom-up along a join tree, with views keyed by join attributes so
 * that D is never materialised. The cardinality constraints of Section 2 (relation
 * sizes, attribute domains) are part of the input: every join or categorical
 * attribute declares its domain [0, domain).
 *
 * Conventions for every call:
 *   - The return value is an int status: LMFAO_OK (0) or a negative LMFAO_ERR_* code.
 *     The message of the last failing call on a context is lmfao_last_error(ctx).
 *     No C++ exception crosses this boundary.
 *   - Strings are NUL-terminated and only read during the call.
 *   - Pointers marked "host" are CPU memory; "device" pointers are CUDA device memory
 *     of the context's device. Nothing is retained after a call returns unless the
 *     call says so (LMFAO_ADOPT_DEVICE, lmfao_fetch results).
 *   - A context is used by one host thread at a time.
 */
#ifndef LMFAO_H
#define LMFAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LMFAO_API __attribute__((visibility("default")))
#else
#define LMFAO_API
#endif

typedef struct lmfao_ctx lmfao_ctx;

/* ---- status codes ------------------------------------------------------------------ */
enum {
  LMFAO_OK = 0,
  LMFAO_ERR_ARG = -1,          /* malformed argument, unknown attribute or relation    */
  LMFAO_ERR_DTYPE = -2,        /* dtype not allowed for the column's role              */
  LMFAO_ERR_KEY_RANGE = -3,    /* a key/categorical value outside [0, domain)          */
  LMFAO_ERR_CYCLIC = -4,       /* the schema has no join tree (GYO reduction fails)    */
  LMFAO_ERR_NOT_PLANNED = -5,  /* lmfao_run / lmfao_fetch before a successful plan/run */
  LMFAO_ERR_OOM = -6,          /* device allocation failed                             */
  LMFAO_ERR_CUDA = -7,         /* a CUDA runtime call failed                           */
  LMFAO_ERR_TIMEOUT = -8,      /* a bounded device wait ran out                        */
  LMFAO_ERR_UNSUPPORTED = -9   /* outside what this engine evaluates (message says why)*/
};

/* ---- relations (Section 2: the database schema with its cardinality constraints) ---- */
enum { LMFAO_I32 = 0, LMFAO_F32 = 1, LMFAO_U8 = 2 };            /* column dtypes */
enum { LMFAO_KEY = 0, LMFAO_CAT = 1, LMFAO_CONT = 2 };          /* column roles  */

typedef struct lmfao_column {
  const char *attr;   /* attribute name; equal names in two relations are joined        */
  int32_t dtype;      /* KEY and CAT: LMFAO_I32; CONT: LMFAO_F32 or LMFAO_U8 (0/1 flags)  */
  int32_t role;       /* LMFAO_KEY (join attribute), LMFAO_CAT, LMFAO_CONT               */
  int64_t domain;     /* KEY and CAT: values lie in [0, domain); ignored for CONT        */
  const void *data;   /* nrows values, host or device memory according to the flags    */
} lmfao_column;

enum {
  LMFAO_HOST = 0,          /* column data are host pointers; copied during the call     */
  LMFAO_DEVICE = 1,        /* column data are device pointers; copied during the call   */
  LMFAO_ADOPT_DEVICE = 2   /* device pointers borrowed until lmfao_destroy: the caller
                              keeps them alive and unchanged                             */
};

/* ---- aggregate batch (Section 2 queries Q1-Q3; Section 3 LR, CART, Rk-means) ---------- */
enum { LMFAO_FN_ID = 0, LMFAO_FN_POW = 1 };  /* f(x) = x, f(x) = x^param (param >= 1) */

typedef struct lmfao_factor {
  const char *attr;   /* a CONT attribute, or a KEY/CAT attribute read as its integer value */
  int32_t fn;         /* LMFAO_FN_ID or LMFAO_FN_POW                                     */
  int32_t param;      /* exponent for LMFAO_FN_POW                                        */
} lmfao_factor;

typedef struct lmfao_aggregate {  /* SUM(prod factors); nfactors == 0 is SUM(1) = COUNT */
  const lmfao_factor *factors;
  int32_t nfactors;
} lmfao_aggregate;

enum { LMFAO_GB_VALUE = 0, LMFAO_GB_BUCKET = 1 };

typedef struct lmfao_groupby {
  const char *attr;          /* VALUE: a KEY or CAT attribute, grouped by its value      */
  int32_t kind;              /* BUCKET: a CONT attribute, grouped by the number of       */
  int32_t nthresholds;       /*   thresholds strictly below x (x == t falls on the <=    */
  const float *thresholds;   /*   side); thresholds ascending, host memory               */
} lmfao_groupby;

enum { LMFAO_LE = 0, LMFAO_LT = 1, LMFAO_GE = 2, LMFAO_GT = 3, LMFAO_EQ = 4, LMFAO_NE = 5 };

typedef struct lmfao_predicate {  /* attr op t, compared on the stored FP32/integer value */
  const char *attr;
  int32_t op;
  float t;
} lmfao_predicate;

/* ---- planning ---------------------------------------------------------------------- */
/* Arithmetic of the path. FP64: the plain FP64 form (every product and sum in FP64).
 * FP32: per-tuple products and per-segment sums in FP32, cross-CTA reductions in FP64,
 * counts exact. SPLIT_BF16: as FP32, with the dense cross-relation contraction on the
 * tensor cores, each FP32 operand split into two BF16 terms (three products, FP32
 * accumulation). A precision this build does not evaluate gives LMFAO_ERR_UNSUPPORTED. */
enum { LMFAO_FP64 = 0, LMFAO_FP32 = 1, LMFAO_SPLIT_BF16 = 2 };
enum {
  LMFAO_PLAN_HEURISTIC = 0,   /* rule-based choices (largest relation as root, ...)        */
  LMFAO_PLAN_EXHAUSTIVE = 1,  /* time every candidate plan on the device, keep the fastest */
  LMFAO_PLAN_LEARNED = 2,     /* rank candidates with the learned cost model (MLP)         */
  LMFAO_PLAN_FORCED = 3       /* use root_rel / segment_rel / mode as given                */
};
/* Root-pass modes: AUTO and FACTORISED use the specialised pass when the plan has at most
 * one inner child of the root (else the generic pass); GENERIC forces the generic pass
 * (per-segment sums, per-tuple accumulation of inner-grouped items); PER_TUPLE evaluates
 * every item per tuple of the root relation. All modes give the same results. */
enum { LMFAO_MODE_AUTO = 0, LMFAO_MODE_FACTORISED = 1, LMFAO_MODE_PER_TUPLE = 2, LMFAO_MODE_GENERIC = 3 };

typedef struct lmfao_plan_opts {
  int32_t precision;        /* LMFAO_FP64 (plain form), LMFAO_FP32, LMFAO_SPLIT_BF16     */
  int32_t planner;          /* LMFAO_PLAN_*                                              */
  int32_t root_rel;         /* FORCED: relation id of the root relation (-1: default)   */
  int32_t segment_rel;      /* FORCED: child of the root whose join key orders the root
                               relation into segments (-1: none, -2: default)            */
  int32_t mode;             /* LMFAO_MODE_*: factorised views or per-tuple evaluation   */
  int32_t autotune;         /* nonzero: time a small set of launch shapes (root-pass work-
                               item length, combine chunk) on the data while planning and
                               keep the fastest; winners are cached in the file
                               LMFAO_TUNE_CACHE (default ~/.cache/lmfao/tiles.txt) by plan
                               shape and device, so the same shape is timed once        */
  const int32_t *join_parent; /* host, nullable: parent relation id per relation (-1 for
                               the tree root) to impose a join tree instead of GYO       */
  const int32_t *query_root;  /* host, nullable: logical root relation per query (-1:
                               heuristic); used by the view-generation layer             */
  const char *cost_model;   /* path of a learned cost model file (LEARNED), or NULL      */
  int32_t combine;          /* 0: automatic; 1: entry-wise combine; 2: prefix-block combine
                               when the plan allows it (results are the same)             */
  int32_t learned_topk;     /* LEARNED: 0 or 1 takes the candidate of least predicted time;
                               k > 1 times the k best-predicted candidates (among those
                               whose checks pass) on the device and keeps the fastest     */
} lmfao_plan_opts;

typedef struct lmfao_plan_info {
  int32_t root_rel;          /* root relation of the physical plan                      */
  int32_t segment_rel;       /* relation whose key forms the segments (-1: none)        */
  int64_t n_segments;        /* segments of the root relation                           */
  int32_t n_views;           /* directional views of the logical plan (after merging)   */
  int32_t n_groups;          /* view groups of the logical plan                          */
  int32_t n_kernels;         /* kernel launches of one lmfao_run                         */
  int32_t mode;              /* mode chosen                                              */
  double predicted_ms;       /* planner's time estimate (-1 if none)                     */
  double plan_ms;            /* host+device time spent planning (incl. reorganisation)   */
  double reorg_ms;           /* of which: reorganising the root relation into segment order
                                (the context keeps that order per root relation and segment
                                key, so a later plan over the same relations reuses it)   */
  int32_t reorg_reused;      /* 1: the segment order of an earlier plan was reused       */
  int32_t n_roots;           /* physical plans (roots) of the batch: 1, or more when no single
                                root determines every query's group-by attributes; root_rel,
                                segment_rel, n_segments and mode then describe the first */
} lmfao_plan_info;

/* ---- results ------------------------------------------------------------------------ */
typedef struct lmfao_result {
  int64_t ngroups;            /* groups with COUNT > 0 (an ungrouped query: always 1)    */
  int32_t ngroupby;           /* group-by attributes of the query                        */
  int32_t naggs;              /* aggregates of the query                                 */
  const int32_t *group_keys;  /* host, ngroups x ngroupby, ascending lexicographic order */
  const int64_t *counts;      /* host, ngroups: COUNT(*) of the group under the filter   */
  const double *sums;         /* host, ngroups x naggs, row-major                        */
} lmfao_result;

/* ==== entry points ==================================================================== */

/* Create a context bound to CUDA device `device`; *out receives the handle. With
 * device == -1 the context is host-only: it takes host relations, batches and plans the
 * logical layer (join tree, query roots, views, groups; lmfao_describe_plan) but runs
 * nothing (lmfao_run returns LMFAO_ERR_NOT_PLANNED). LMFAO_ERR_CUDA if the device is
 * unusable. */
LMFAO_API int lmfao_create(struct lmfao_ctx **out, int device);

/* Free every device and host resource of the context (adopted columns are not freed). */
LMFAO_API int lmfao_destroy(struct lmfao_ctx *ctx);

/* Message of the last failing call on ctx ("" if none); valid until the next call. */
LMFAO_API const char *lmfao_last_error(const struct lmfao_ctx *ctx);

/* Add a relation (Section 2 schema). `cols` describes `ncols` columns of `nrows` values.
 * KEY/CAT values outside [0, domain) give LMFAO_ERR_KEY_RANGE (checked here).
 * Relations are immutable once loaded; loading invalidates a previous plan.
 * *rel_id receives the relation's id (0, 1, ... in load order). */
LMFAO_API int lmfao_load_relation(struct lmfao_ctx *ctx, const char *name, int64_t nrows,
                        const lmfao_column *cols, int ncols, uint32_t flags, int *rel_id);

/* Add one query of the batch: `naggs` aggregates sharing the group-by attributes `gb`
 * and the conjunctive filter `filters` (Section 2 queries; Section 3 aggregates).
 * Unknown attributes give LMFAO_ERR_ARG. *query_id receives 0, 1, ... in call order.
 * Adding a query invalidates a previous plan. */
LMFAO_API int lmfao_add_batch(struct lmfao_ctx *ctx, const lmfao_aggregate *aggs, int naggs,
                    const lmfao_groupby *gb, int ngb, const lmfao_predicate *filters,
                    int nfilters, int *query_id);

/* Remove all queries (relations stay loaded). */
LMFAO_API int lmfao_clear_batch(struct lmfao_ctx *ctx);

/* Build the plan for the current batch (Fig. 1 view generation and multi-output
 * layers): join tree (GYO, LMFAO_ERR_CYCLIC when there is none), per-query roots,
 * directional views and their merging, view groups; then the physical plan: the root
 * relation reorganised as a trie ordered by its segment key, view layouts, kernel
 * sequence. opts may be NULL (heuristic FP32). info may be NULL. May launch device
 * work (reorganisation, autotuning) on the context's internal stream and waits for it.
 * For a root relation of at least 2^20 tuples the root pass is generated for the batch
 * and compiled with NVRTC (Fig. 1's code generation; about 0.3 s per new shape, cached
 * for the life of the process; a shape outside the generators uses the built-in kernel).
 * A group-by attribute of a non-root relation must be determined by the key of that
 * relation's view toward the root; this is checked on the loaded data while planning. The
 * heuristic planner then moves the root (largest relations first) and a forced root that
 * fails gives LMFAO_ERR_UNSUPPORTED.
 * The views of relations with unique keys and no children are generated the same way.
 * Environment (for comparisons and tests; every form computes the same aggregates):
 * LMFAO_CODEGEN=0 never generates (root pass and views), =1 generates the root pass at any
 * size; LMFAO_ROOT_LANES=1 generates the one-tuple-per-lane layout of the root pass;
 * LMFAO_NO_PROJECTION_COMBINE selects the entry-wise combine where the projection combine
 * would run, LMFAO_PROJECTION=stream|kernels its streaming or per-projection form;
 * LMFAO_COMBINE=single keeps the single-kernel block combine, =general the term-by-term
 * two-kernel form, =dense the dense form without the cp.async pipeline;
 * LMFAO_COMBINE_CHUNK sets the block combine's chunk of segments. */
LMFAO_API int lmfao_plan(struct lmfao_ctx *ctx, const lmfao_plan_opts *opts, lmfao_plan_info *info);

/* Candidate physical plans of the current batch (root relation, segment relation, root
 * pass, combine) for training a cost model: cand (host, cap x 4 int32: root_rel,
 * segment_rel, mode, combine -- usable as FORCED plan options) and feats (host, cap x nfeat
 * floats: the features the LEARNED planner feeds to its model). Either may be NULL.
 * *n receives the number of candidates, *nfeat the feature count. */
LMFAO_API int lmfao_plan_candidates(struct lmfao_ctx *ctx, const lmfao_plan_opts *opts, int32_t *cand, float *feats,
                                    int cap, int *n, int *nfeat);

/* Evaluate the planned batch asynchronously on `stream` (a cudaStream_t; NULL = the
 * legacy default stream). All work (view kernels, root pass, contraction,
 * finalisation) is enqueued on that stream; device-side failures are latched and
 * reported by the next lmfao_fetch. */
LMFAO_API int lmfao_run(struct lmfao_ctx *ctx, void *stream);

/* Results of query `query_id` from the last lmfao_run: waits for that run's stream,
 * copies the results to host memory owned by the context (valid until the next
 * lmfao_run, lmfao_plan or lmfao_destroy) and fills *out. */
LMFAO_API int lmfao_fetch(struct lmfao_ctx *ctx, int query_id, lmfao_result *out);

/* Copy of the dense device result of query `query_id` into caller memory: counts
 * (int64, one per dense group cell) and sums (double, cells x naggs), where the dense
 * cells enumerate the group-by domains in mixed radix (first attribute most
 * significant). `counts`/`sums` are device pointers (either may be NULL), filled
 * asynchronously on `stream` after the last lmfao_run. *ncells receives the number of
 * cells (may be queried with both pointers NULL). */
LMFAO_API int lmfao_result_device(struct lmfao_ctx *ctx, int query_id, int64_t *counts, double *sums,
                        int64_t *ncells, void *stream);

/* The plan's result state: every result of the batch (all queries) lives in two device
 * arrays of a fixed layout that depends only on the batch and the attribute domains,
 * not on the data or the physical plan: *counts (int64: per dense group cell the COUNT
 * and the integral sums) and *sums (double: the other sums), with *ncounts and *nsums
 * elements. Every entry is a sum over the tuples of the join, so when the rows of one
 * relation are split into disjoint shards, each evaluated by its own context with the
 * same batch (one GPU per shard), the element-wise sum of the shards' arrays is the
 * state of the whole relation (the merge of a data-parallel run, Section 2: the join
 * distributes over a partition of any of its relations). The pointers are owned by the
 * context, valid until the next lmfao_plan or lmfao_destroy; lmfao_run overwrites them on
 * its stream, and lmfao_fetch / lmfao_result_device read them, so a caller that sums the
 * arrays in place (an all-reduce) orders that after the run on the run's stream and
 * before the fetch. Either pointer argument may be NULL. ERR_NOT_PLANNED without a plan. */
LMFAO_API int lmfao_result_state(struct lmfao_ctx *ctx, int64_t **counts, int64_t *ncounts, double **sums,
                                 int64_t *nsums);

/* Text (JSON) description of the current plan into buf (at most len bytes, NUL-
 * terminated); *needed receives the full length + 1. The logical part lists the join
 * tree, the root of every query, the directional views V_{u->v} after merging and the
 * view groups with their dependencies (Fig. 2); the physical part lists the kernels. */
LMFAO_API int lmfao_describe_plan(struct lmfao_ctx *ctx, char *buf, size_t len, size_t *needed);

/* CART split variances (Section 3, decision trees) of bucketed queries, in FP64 on the
 * device: each query q in qids (host array of n ids) must have exactly one BUCKET
 * group-by with B = nthresholds + 1 buckets (the same B for all) and exactly three
 * aggregates, COUNT, SUM(y) and SUM(y^2) of one value attribute y, in any order (y^2
 * written as y^2 or y * y); anything else gives LMFAO_ERR_ARG. For every threshold
 * k < B - 1 the left fragment is buckets 0..k and the right the rest; VARIANCE(T) =
 * SUM(y^2) - SUM(y)^2 / |T| (0 if T is empty). `out` (device, n x (B-1) x 2 doubles:
 * left, right) is written asynchronously on `stream`. Waits for the last run and returns
 * the status lmfao_fetch would give for its device-side failures. */
LMFAO_API int lmfao_cart_variances(struct lmfao_ctx *ctx, const int *qids, int n, double *out, void *stream);

/* One node of a regression tree grown by lmfao_cart_tree (nodes in heap order: the children
 * of node i are 2i + 1 (left, x <= threshold) and 2i + 2 (right, x > threshold)). */
typedef struct lmfao_cart_node {
  int32_t active;      /* 1: the node was evaluated (every ancestor split)                   */
  int32_t feature;     /* index into features[] of the chosen split, -1: no valid split     */
  float threshold;     /* the split: left x <= threshold, right x > threshold               */
  double score;        /* VARIANCE(left) + VARIANCE(right) of the chosen split             */
  int64_t count;       /* tuples of the join that reach the node                            */
  double sum_y, sum_y2;  /* SUM(y), SUM(y^2) over those tuples                              */
} lmfao_cart_node;

/* Grow a regression tree (Section 3, decision trees) over the natural join of the loaded
 * relations: levels 0 .. depth-1, every node of a level evaluated in one batch (one query
 * per node and feature: COUNT, SUM(y), SUM(y^2) GROUP BY the feature's bucket, filtered by
 * the node's path of split predicates), one plan and run per level (the reorganised root
 * relation is reused across levels) and the best split of every node chosen on the device:
 * the least VARIANCE(left) + VARIANCE(right) over the features' thresholds with both sides
 * non-empty, ties to the lower feature index, then the lower threshold. `target` is a CONT
 * attribute (y); `features` (host, nfeatures names) CONT attributes; `thresholds` (host)
 * their ascending thresholds concatenated, nthresholds[f] of them for feature f (at most 31
 * per feature); depth in [1, 5]. opts as for lmfao_plan (NULL: FP32, heuristic). nodes
 * (host, 2^depth - 1 entries) receives the tree; level_ms (host, depth x 2 doubles or NULL)
 * the host time of planning and of the run plus split selection per level. The context's
 * batch is replaced (cleared on return); relations stay loaded. */
LMFAO_API int lmfao_cart_tree(struct lmfao_ctx *ctx, const char *target, const char *const *features, int nfeatures,
                              const float *thresholds, const int32_t *nthresholds, int depth,
                              const lmfao_plan_opts *opts, lmfao_cart_node *nodes, double *level_ms);

/* Ridge linear regression over the join (Section 3, linear regression) from the aggregates
 * of query `query_id` of the last run: the model theta_0 + sum_f theta_f x_f for the target y,
 * minimising J(theta) = 1/(2|D|) SUM_D (theta^T x - y)^2 + lambda/2 |theta|^2 with x = (1,
 * x_1 .. x_d). J and its gradient need only Sigma = SUM x x^T, SUM x y and SUM y^2, which the
 * query must hold (ungrouped, unfiltered; COUNT, SUM(x_f), SUM(y), SUM(x_f x_g), SUM(x_f y),
 * SUM(y^2) in any order, as the ridge batch of Section 3 does): a missing one gives
 * LMFAO_ERR_ARG naming it. method LMFAO_RIDGE_CLOSED_FORM solves (Sigma_xx/|D| + lambda I)
 * theta = Sigma_xy/|D| by Cholesky; LMFAO_RIDGE_BGD runs `iters` batch gradient steps of size
 * `step` from theta = 0. Computed in FP64 on the device. theta (host, nfeatures + 1: intercept
 * first), *loss = J(theta) and *grad_norm = |grad J(theta)| (either may be NULL). At most 126
 * features. */
enum { LMFAO_RIDGE_CLOSED_FORM = 0, LMFAO_RIDGE_BGD = 1 };
LMFAO_API int lmfao_ridge_fit(struct lmfao_ctx *ctx, int query_id, const char *target, const char *const *features,
                              int nfeatures, double lambda, int method, int iters, double step, double *theta,
                              double *loss, double *grad_norm);

/* COUNT GROUP BY gb over the natural join of the loaded relations, with the groups kept in
 * hash tables in device memory: the group-bys of Rk-means (Section 3), SUM(1) GROUP BY X_j
 * over the values of one attribute (step 1) and SUM(1) GROUP BY C_1, ..., C_n over the cells
 * of a grid of cluster intervals (step 3), whose key spaces are too large for the dense
 * result cells of a batch. Each group attribute is VALUE (a KEY or CAT attribute by its value;
 * a CONT attribute by its FP32 value, reported as its 32-bit pattern; a U8 one by its value)
 * or BUCKET (a CONT attribute by the number of thresholds strictly below it). The product of
 * the attributes' domains (2^32 for an FP32 value) must stay below 2^62 (else
 * LMFAO_ERR_UNSUPPORTED), and attributes of non-root relations must be determined by the join
 * key toward the root. keys (device, cap x ngb int32 codes) and counts (device, cap int64)
 * receive min(groups, cap) groups in no particular order; *ngroups (host) the number of
 * groups. Independent of the batch and plan; synchronous on the context's stream. */
LMFAO_API int lmfao_group_count(struct lmfao_ctx *ctx, const lmfao_groupby *gb, int ngb, int64_t cap, int32_t *keys,
                                int64_t *counts, int64_t *ngroups);

/* Allocation-free variant of lmfao_cart_variances (same arguments, same results), for
 * callers that cannot allocate device memory when they ask for split variances: a host
 * framework that gives the engine a fixed device-memory budget through its own caching
 * allocator, or a tree-building loop that must not pay the device-wide synchronisation
 * cudaMalloc / cudaFree can cause. The paper has no counterpart of this call; it exists
 * for those callers only. The per-query descriptors live in a fixed device array of
 * LMFAO_NOALLOC_MAX_QUERIES entries (192 KiB, held on every device that loads the
 * library until the process exits); n above that limit gives LMFAO_ERR_ARG. The first
 * call on a device looks up the array's device address, so make that first call before
 * any stream capture. Each call fills the descriptors on the host under a process-wide
 * lock and copies them into the array with cudaMemcpyAsync on `stream` before its kernel,
 * so calls from several host threads do not mix their descriptors; but all calls on a
 * device share the one device array, so calls whose work overlaps on the GPU (other
 * streams, other contexts) race on it. No cudaMalloc, cudaFree or other allocating
 * routine is called. */
#define LMFAO_NOALLOC_MAX_QUERIES 4096
LMFAO_API int lmfao_cart_variances_noalloc(struct lmfao_ctx *ctx, const int *qids, int n, double *out,
                                           void *stream);

/* ---- learned cost model (planner) -----------------------------------------------------
 * A 3-layer perceptron of width 64 over plan features predicts log run time of a plan
 * (the planner's "find roots" and grouping choices of Fig. 1 are ranked by it). Parameters
 * are one FP32 device buffer of lmfao_mlp_param_count(d) floats: W1 (d x 64, row-major),
 * b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1). All pointers are device memory; work is
 * enqueued on `stream`. d must be in [1, 256]. */
LMFAO_API int64_t lmfao_mlp_param_count(int d);
/* y[i] = MLP(x[i, :]) for n samples (x: n x d). h1, h2 (n x 64 each) receive the hidden
 * activations when non-NULL (needed by lmfao_mlp_backward). */
LMFAO_API int lmfao_mlp_forward(const float *x, int n, int d, const float *params, float *h1, float *h2, float *y,
                                void *stream);
/* loss = mean((y - t)^2) into *loss (device float) and gy[i] = 2 (y[i] - t[i]) / n. */
LMFAO_API int lmfao_mlp_loss(const float *y, const float *t, int n, float *gy, float *loss, void *stream);
/* grad = d(sum_i gy[i] * y[i]) / d(params) from the activations of lmfao_mlp_forward. */
LMFAO_API int lmfao_mlp_backward(const float *x, int n, int d, const float *params, const float *h1,
                                 const float *h2, const float *gy, float *grad, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected for step >= 1). */
LMFAO_API int lmfao_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t np, int step, float lr,
                             void *stream);

/* Timings of the last lmfao_run measured with CUDA events around each kernel (host
 * array of at most cap doubles, milliseconds, in launch order; names via
 * lmfao_kernel_name). Waits for the run's stream. *n receives the number of kernels. */
LMFAO_API int lmfao_kernel_times(struct lmfao_ctx *ctx, double *ms, int cap, int *n);
LMFAO_API const char *lmfao_kernel_name(struct lmfao_ctx *ctx, int i);

/* Turn per-kernel event timing of lmfao_run on (1) or off (0, default). */
LMFAO_API int lmfao_set_profiling(struct lmfao_ctx *ctx, int on);

#ifdef __cplusplus
}
#endif
#endif /* LMFAO_H */
