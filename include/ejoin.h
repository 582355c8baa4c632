/*
 * ejoin.h -- C ABI of the GB300 (sm_103a) tensor-join hot path of the
 * context-enhanced E-join ("Optimizing Context-Enhanced Relational Joins",
 * arXiv 2312.01476).
 *
 * The operator (Sec. III-C, Eq. (E-theta-Join)):
 *
 *     R join_{E,mu,theta} S  =  sigma_theta( E_mu(R) x E_mu(S) )
 *
 * with theta = selR(r) and selS(s) and cos(r, s) >= eps, where cos is
 * Sec. III-A, Eq. (Cosine Similarity).  The embeddings E_mu(R), E_mu(S) are
 * given as FP32 row-major matrices (the embedding model itself is out of
 * scope).  Evaluation follows the tensor formulation of Sec. IV-C: the rows
 * are normalised once (cosine equals the dot product of normalised rows),
 * the similarity matrix D = R S^T is formed block by block (Eq. Block Matrix
 * Dot Product Decomposition; Sec. V-B: D is never materialised, only one
 * tile at a time lives on chip), and the pairs passing the threshold are
 * mapped back to tuple ids through the tile offsets (Sec. IV-C, late
 * materialisation).  Relational predicates are pushed below the vector work
 * (Eq. (E-Selection); Sec. VI-E pre-filter).
 *
 * Conventions for every entry point:
 *   - Every function returns an ejoin_status; nothing aborts and no C++
 *     exception crosses the ABI.  ejoin_strerror() gives the text.
 *   - Unless stated otherwise, pointers named d_* or documented as "device"
 *     are CUDA device pointers owned by the caller; all work is enqueued on
 *     the context's stream in order.
 *   - Pair ids are 0-based row numbers of the ORIGINAL relations (before any
 *     selection).  A self-join (R and S describe the same matrix and the same
 *     selection) yields every ordered pair, including (i, i).
 *   - Result: every pair whose FP64 similarity differs from eps by at least
 *     1e-5 is in the result iff sim >= eps; each emitted similarity is within
 *     1e-5 of the FP64 value (it is re-scored in FP32 from the input rows,
 *     in FP64 when it lies within fp64_band of eps).  Order is unspecified
 *     unless EJOIN_FLAG_SORT asks for ascending (i, j).
 *   - A context holds the workspace and statistics of its calls, so calls on
 *     one context must not overlap (from several host threads at once).
 *     Separate contexts may be used from separate threads; each calls
 *     cudaSetDevice for its device and restores the caller's device.
 */
#ifndef EJOIN_H
#define EJOIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ejoin_status {
    EJOIN_OK = 0,
    EJOIN_EINVAL = 1,       /* bad argument (null pointer, d mismatch, d out of range, ...) */
    EJOIN_ENOMEM = 2,       /* device allocation failed */
    EJOIN_EOVERFLOW = 3,    /* more pairs than the caller's capacity; count holds the total */
    EJOIN_ENONFINITE = 4,   /* an input row holds NaN or Inf */
    EJOIN_ECUDA = 5,        /* a CUDA runtime/driver call failed (no device, launch error, ...) */
    EJOIN_ETIMEOUT = 6,     /* a bounded device-side wait gave up; results are invalid */
    EJOIN_EUNSUPPORTED = 7  /* precision or shape not supported on this device */
} ejoin_status;

/* Arithmetic of the bulk similarity contraction.  Every precision is followed
 * by an exact re-score of the candidates within a guard band of eps, so all
 * of them return the same result set (see the conventions above). */
typedef enum ejoin_prec {
    EJOIN_F32 = 0,      /* FP32 CUDA-core contraction (the plain FP32 path) */
    EJOIN_BF16 = 1,     /* tcgen05 kind::f16 on BF16 rows, FP32 accumulation in TMEM */
    EJOIN_FP8_E4M3 = 2, /* tcgen05 kind::f8f6f4 on e4m3 rows with per-row FP32 scales */
    EJOIN_TF32 = 3      /* tcgen05 kind::tf32 on FP32 rows, FP32 accumulation in TMEM */
} ejoin_prec;

/* ejoin_config.flags */
#define EJOIN_FLAG_COUNT_ONLY 0x1u /* count the pairs, store none (a "count pass") */
#define EJOIN_FLAG_TIMING     0x2u /* record CUDA events around each stage (ejoin_last_stats) */
#define EJOIN_FLAG_FUSED      0x4u /* tensor-core precisions: run the re-score as extra warps of the
                                      contraction kernel (one launch; needs 16-byte aligned rows,
                                      d % 4 == 0 and a caller-supplied result buffer).  Off by default:
                                      on GB300 the separate re-score kernel, with the whole GPU behind it,
                                      is faster on candidate-dense joins */

#define EJOIN_FLAG_NO_SYMMETRY 0x8u /* evaluate a self-join over the full square of pairs.  By default a
                                      self-join on the tensor cores contracts only the 256-row block
                                      pairs on and above the diagonal and writes every pair (i, j),
                                      i != j, in both orders; the result is the same set */
#define EJOIN_FLAG_HOST_COPY  0x10u /* ejoin_threshold_host: copy the inputs to the device whole even when
                                       the kernels could read them in place (see there) */
#define EJOIN_FLAG_GATHER_RESCORE 0x20u /* re-score the candidates in emission order, gathering both FP32 rows of
                                           each from global memory.  By default, for d % 4 == 0, d <= 1024,
                                           16-byte aligned rows and joins of at least 2^27 pairs (before
                                           selection), the candidates are first bucketed by panels of
                                           consecutive R rows and each panel's rows are staged in shared memory
                                           once; both give the same pairs and similarities */
#define EJOIN_FLAG_PANEL_RESCORE 0x80u /* the panel-ordered re-score at any join size (where the rows allow
                                          it); without it smaller joins gather in emission order, which
                                          needs one synchronisation less per call */
#define EJOIN_FLAG_SORT       0x40u /* ejoin_threshold, ejoin_threshold_host, ejoin_eselect and
                                       ejoin_threshold_pruned return their records sorted by (i, j)
                                       ascending (a device radix sort after the join; the call
                                       synchronises once more) instead of in no particular order */

typedef struct ejoin_config {
    int32_t device;          /* CUDA device ordinal */
    void *stream;            /* cudaStream_t for all work; NULL = the legacy default stream */
    int32_t prec;            /* ejoin_prec */
    float band;              /* guard band around eps for re-scoring; < 0: the rigorous default
                                1.25 (2u + u^2 + 2 g + 8 * 2^-24) for prec and d, with g = kp 2^-24
                                (FP32 accumulation over the kp padded columns) and u = 2^-8 (BF16),
                                2^-10 (TF32) or, for e4m3, 2^-4 + 2^-10 sqrt(kp) / 448 (u = 0 for
                                the FP32 CUDA-core path) */
    float fp64_band;         /* candidates with |sim32 - eps| < fp64_band are re-scored in FP64;
                                < 0: default 2e-5 */
    uint64_t capacity_hint;  /* initial candidate-buffer size in pairs (0: 1 << 20); grows on demand */
    uint32_t flags;          /* EJOIN_FLAG_* */
    uint64_t timeout_cycles; /* bound on every device-side spin-wait, in SM clock cycles
                                (0: 2^31, about one second) */
    int32_t group_m;         /* tensor-core contraction raster: row tiles per group (0: sized so
                                that one group's FP32 rows take about 40 MB) */
} ejoin_config;

/* A relation: n rows of d FP32 values, row r at x + r * ld (ld >= d).
 * Device memory for ejoin_threshold/ejoin_normalize; host memory for
 * ejoin_threshold_host.  1 <= d <= 4096 and n < 2^31 - 256. */
typedef struct ejoin_rel {
    const float *x;
    int64_t n;
    int32_t d;
    int64_t ld;
} ejoin_rel;

/* Relational selection pushed below the join (Sec. III-C, Eq. (Selection) and
 * Eq. (E-Selection)): keep row r iff attr[r] <op> c, and, when bits is not
 * NULL, bit (r % 32) of bits[r / 32] is set.  attr may be NULL (bits only).
 * A NULL ejoin_sel* keeps every row.  Arrays have n entries (bits: ceil(n/32)). */
typedef enum ejoin_op { EJOIN_LT = 0, EJOIN_LE = 1, EJOIN_GT = 2, EJOIN_GE = 3, EJOIN_EQ = 4, EJOIN_NE = 5 } ejoin_op;
typedef struct ejoin_sel {
    const int32_t *attr;
    int32_t op;
    int32_t c;
    const uint32_t *bits;
} ejoin_sel;

/* One result tuple: the pair of original row ids and its similarity (Sec. IV-C:
 * "tuples of offsets"). */
typedef struct ejoin_pair {
    uint32_t i;
    uint32_t j;
    float sim;
} ejoin_pair;

/* Result buffer.  If d_pairs == NULL on entry the library allocates it (sized to
 * the candidate count) and ejoin_pairs_free releases it; otherwise the caller's
 * buffer of `capacity` records is used.  d_count (device, optional) receives the
 * exact total; count (host) receives it too when the call returns. */
typedef struct ejoin_pairs {
    ejoin_pair *d_pairs;
    uint64_t capacity;
    uint64_t *d_count;
    uint64_t count;
} ejoin_pairs;

typedef struct ejoin_ctx ejoin_ctx;

/* Per-call statistics of the last ejoin_threshold / ejoin_threshold_host / ejoin_topk call
 * (top-k: candidates = pairs kept by the second pass, pairs = records written). */
typedef struct ejoin_stats {
    uint64_t n_sel_r, n_sel_s;  /* rows kept by the selections */
    uint64_t candidates;        /* pairs at or above eps - band in the bulk precision (a symmetric
                                   self-join counts each unordered pair once) */
    uint64_t fp64_rescored;     /* candidates re-scored in FP64 */
    uint64_t pairs;             /* result pairs */
    uint64_t launches;          /* kernels launched by the call */
    float band;                 /* guard band used */
    float ms_select, ms_normalize, ms_contract, ms_rescore, ms_total; /* FLAG_TIMING only; with the fused
                                                                         kernel ms_contract covers both */
    float ms_h2d, ms_d2h;       /* ejoin_threshold_host only, FLAG_TIMING only */
    int32_t contract_retries;   /* candidate-buffer regrowths */
    int32_t fused;              /* 1 if the re-score ran fused into the contraction */
    uint64_t h2d_bytes;         /* ejoin_threshold_host only: bytes read from host memory (copied, or read
                                   in place by the kernels) */
    int32_t host_in_place;      /* ejoin_threshold_host only: 1 if the kernels read the host buffers in place */
    int32_t reserved;
} ejoin_stats;

/* Create a context on cfg->device (made current for the call).  cfg may be
 * NULL (device 0, default stream, BF16).  *out receives the context. */
ejoin_status ejoin_create(ejoin_ctx **out, const ejoin_config *cfg);

/* Release the context, its workspace and events.  NULL is ignored. */
void ejoin_destroy(ejoin_ctx *ctx);

/* Row normalisation with selection pushdown (Sec. IV-C: cosine is the dot
 * product of normalised rows; Eq. (E-Selection)).  For each kept row r, in
 * ascending order c = 0, 1, ..., writes y = x_r / ||x_r|| (0 for a zero row)
 * in `prec`'s storage format to d_out + c * ld_out (elements; ld_out >= the
 * padded dimension ejoin_padded_dim(prec, d), padding zero-filled),
 * 1/||x_r|| to d_inv_norm[c] (optional), the e4m3 scale to d_scale[c]
 * (required for EJOIN_FP8_E4M3, else ignored), r to d_ids[c] (optional), and
 * the number of kept rows to *d_n_sel (device int64).  Non-finite input sets
 * the context's error word; the next synchronising call reports ENONFINITE.
 * Storage: F32 and TF32 float, BF16 __nv_bfloat16, FP8 __nv_fp8_e4m3. */
ejoin_status ejoin_normalize(ejoin_ctx *ctx, ejoin_rel in, const ejoin_sel *sel, int32_t prec,
                             void *d_out, int64_t ld_out, float *d_inv_norm, float *d_scale,
                             uint32_t *d_ids, int64_t *d_n_sel);

/* Padded row length (elements) used for `prec` at dimension d. */
int64_t ejoin_padded_dim(int32_t prec, int32_t d);

/* The threshold E-join of R and S on the device (Sec. III-C, Eq. (E-theta-Join);
 * tensor formulation Sec. IV-C; tiled, memory-bounded evaluation Sec. V-B).
 * R.x, S.x, the selections' arrays and out->d_pairs / out->d_count are device
 * pointers.  Synchronises the context stream before returning (the pair count
 * is read back).  EJOIN_EOVERFLOW: out->count holds the exact total and the
 * first out->capacity records are valid; retry with a larger buffer. */
ejoin_status ejoin_threshold(ejoin_ctx *ctx, ejoin_rel R, ejoin_rel S, float eps,
                             const ejoin_sel *selR, const ejoin_sel *selS, ejoin_pairs *out);

/* Same operator with HOST inputs and a HOST result buffer: R.x, S.x, the
 * selections' arrays and h_pairs are host pointers; *count receives the total
 * (EOVERFLOW as above).  When every input buffer is device-accessible host
 * memory (pinned, e.g. cudaHostAlloc or cudaHostRegister), the selection
 * kernels read the attribute columns in place and the normalisation pass reads
 * only the kept rows in place, copying them to the device for the re-score: the
 * relational predicate is pushed below the host-to-device transfer (Sec. VI-E
 * pre-filter), and only the kept rows cross the link.  Otherwise (pageable
 * memory, or EJOIN_FLAG_HOST_COPY) the inputs are copied whole first.  On
 * the in-place route a device-accessible h_pairs is written by the re-score
 * directly; otherwise the pairs are copied back to it. */
ejoin_status ejoin_threshold_host(ejoin_ctx *ctx, ejoin_rel R, ejoin_rel S, float eps,
                                  const ejoin_sel *selR, const ejoin_sel *selS,
                                  ejoin_pair *h_pairs, uint64_t capacity, uint64_t *count);

/* The top-k join condition (Sec. VI-E, the "top-k" vector join predicate; the
 * paper evaluates k = 1 and k = 32), 1 <= k <= 32: for every row i of R kept
 * by selR, the kk = min(k, kept S rows) rows j of S kept by selS of largest
 * cosine similarity, in descending similarity, ties to the smaller j.  Writes
 * kk records (i, j, sim) per kept R row, the rows in ascending i, each row's
 * records consecutive (record t of the r-th kept row at r * kk + t).  Device
 * pointers as for ejoin_threshold; out->d_pairs NULL: the library allocates
 * kk records per kept R row.  Evaluation: two passes of the tensor-core
 * contraction (per row, a lower bound of its k-th largest bulk similarity,
 * then every column within 2 * band of it, which holds the exact top k) and
 * an FP32 re-score of those candidates; the t-th record's FP64 similarity is
 * within 1e-5 of the row's t-th largest, and sim is its FP32 cosine.  ctx
 * must use BF16, e4m3 or TF32 (F32: EJOIN_EUNSUPPORTED); k outside [1, 32]:
 * EJOIN_EINVAL.  Synchronises.  EOVERFLOW as above. */
ejoin_status ejoin_topk(ejoin_ctx *ctx, ejoin_rel R, ejoin_rel S, int32_t k, const ejoin_sel *selR,
                        const ejoin_sel *selS, ejoin_pairs *out);

/* ejoin_topk with k = 1: one record per kept R row. */
ejoin_status ejoin_top1(ejoin_ctx *ctx, ejoin_rel R, ejoin_rel S, const ejoin_sel *selR,
                        const ejoin_sel *selS, ejoin_pairs *out);

/* ℰ-selection of R against a batch of query vectors (Sec. III-C, Eq.
 * (ℰ-Selection), with a cosine predicate per query; cost one scan of R,
 * Sec. IV-A, Eq. (ℰ-Selection Cost)): every pair (i, q) with selR(i) and
 * cos(R_i, Q_q) >= eps, written as {i, q, sim} (j is the query's row in Q).
 * R.x, Q.x, the selection's arrays and out as for ejoin_threshold (device
 * pointers; out->d_pairs NULL: the library allocates).  Q may hold any number
 * of rows (processed 64 at a time).  The scan is a TF32 tensor-core product
 * of R's FP32 rows with the normalised queries, the row norms taken from the
 * same tiles; the guard band of TF32 (or the context's band) selects the
 * candidates, which the FP32 re-score (and its accurate tier near eps)
 * decides, so the result obeys the same rule as ejoin_threshold: exact
 * outside |sim - eps| < 1e-5, sims within 1e-5.  The context's precision is
 * not used.  Without selR, with R.x 16-byte aligned and R.ld % 4 == 0, R is
 * read in place once per 64 queries; otherwise the kept rows are compacted
 * and normalised first.  For batches of hundreds of queries or more,
 * ejoin_threshold(R, Q, eps, selR, NULL) reads R once for all of them and is
 * the faster call.  Synchronises; EOVERFLOW as for ejoin_threshold. */
ejoin_status ejoin_eselect(ejoin_ctx *ctx, ejoin_rel R, const ejoin_sel *selR, ejoin_rel Q, float eps,
                           ejoin_pairs *out);

/* Release a result buffer that the library allocated. */
ejoin_status ejoin_pairs_free(ejoin_ctx *ctx, ejoin_pairs *pairs);

/* ---------------------------------------------------------------------------
 * Batched joins: many independent E-joins (each the operator above, with its
 * own eps and its own, possibly very different, sizes) in one persistent
 * tensor-core launch.  The rows of all jobs' R and S are normalised into two
 * concatenated operands; a device job table maps the global tile space onto
 * (job, row tile, column tile), so tiles of every job share one persistent
 * grid (the tiles of different jobs are independent blocks of the
 * decomposition of Sec. IV-C, Eq. (Block Matrix Dot Product Decomposition)).
 * Selection predicates per job: ejoin_batch_create_sel.
 * ------------------------------------------------------------------------- */
typedef struct ejoin_job {
    ejoin_rel R;  /* device rows of this job's R (all jobs of a batch share d) */
    ejoin_rel S;  /* device rows of this job's S */
    float eps;    /* this job's similarity threshold */
} ejoin_job;

/* The selections of one job of a batch (Sec. III-C, Eq. (E-Selection); the pre-filter of Sec. VI-E): the R
 * and S predicates of ejoin_threshold (device attr / bits arrays of that job's rows).  A side whose attr and
 * bits are both NULL keeps every row. */
typedef struct ejoin_job_sel {
    ejoin_sel R;
    ejoin_sel S;
} ejoin_job_sel;

/* One result record of a batched join: job index, original row ids, similarity. */
typedef struct ejoin_batch_pair {
    uint32_t job;
    uint32_t i;
    uint32_t j;
    float sim;
} ejoin_batch_pair;

typedef struct ejoin_batch ejoin_batch;

/* ejoin_batch_create flags */
#define EJOIN_BATCH_GRAPH    0x1u /* capture the whole run in a CUDA graph (runs replay it) */
#define EJOIN_BATCH_AUTOTUNE 0x2u /* time candidate raster widths once per size class and keep the fastest
                                     (cached per process, and in the file named by EJOIN_TUNE_FILE) */

typedef struct ejoin_batch_stats {
    int32_t n_jobs;
    int64_t total_tiles;
    int64_t rows_r, rows_s;
    int32_t group_m;      /* raster width in use */
    int32_t graph;        /* 1 if runs replay a CUDA graph */
    uint64_t candidate_capacity, pair_capacity;
    float band;
    float ms_normalize, ms_contract, ms_rescore;  /* stages of one eager run timed when the plan was made */
} ejoin_batch_stats;

/* Plan a batch over the jobs' device inputs (the pointers are captured: the
 * plan reads whatever those rows hold when it runs).  Runs the pipeline once
 * to size the candidate and result buffers (synchronises), optionally
 * autotunes, optionally captures a CUDA graph.  ctx must use BF16, e4m3 or
 * TF32.  A later run whose counts exceed the sized buffers reports
 * EJOIN_EOVERFLOW from ejoin_batch_wait (re-create the plan). */
ejoin_status ejoin_batch_create(ejoin_ctx *ctx, const ejoin_job *jobs, int32_t n_jobs, uint32_t flags,
                                ejoin_batch **out);

/* ejoin_batch_create with per-job selections: sels[j] holds job j's predicates (sels == NULL: none).  Every
 * run evaluates them on the device before the normalisation: each job's kept rows are compacted in order,
 * and the job table, the tile counts and the re-score's sort buckets are rebuilt from the kept counts, so
 * only kept rows are normalised and contracted, and a replayed graph follows whatever the attribute arrays
 * hold when it runs (their pointers are captured like the rows').  Records carry original row ids.  The
 * buffers are sized from the rows kept when the plan is made; a later run that finds more candidates or
 * pairs than fit reports EJOIN_EOVERFLOW from ejoin_batch_wait.  EJOIN_EINVAL for an unknown op. */
ejoin_status ejoin_batch_create_sel(ejoin_ctx *ctx, const ejoin_job *jobs, const ejoin_job_sel *sels, int32_t n_jobs,
                                    uint32_t flags, ejoin_batch **out);

/* Enqueue one run on the context's stream (a graph launch when captured); no host synchronisation. */
ejoin_status ejoin_batch_run(ejoin_batch *batch);

/* Wait for the enqueued runs; *count = result pairs of the last run. */
ejoin_status ejoin_batch_wait(ejoin_batch *batch, uint64_t *count);

/* Device buffer holding the last run's records (valid after ejoin_batch_wait). */
ejoin_status ejoin_batch_result(const ejoin_batch *batch, const ejoin_batch_pair **d_pairs, uint64_t *capacity);

ejoin_status ejoin_batch_info(const ejoin_batch *batch, ejoin_batch_stats *out);

/* Release the plan (synchronises its device; does not use the context, so it may come after ejoin_destroy). */
void ejoin_batch_destroy(ejoin_batch *batch);

/* ---------------------------------------------------------------------------
 * Learned tile pruning.  The paper has no learned component; this is an
 * extension of the tensor join that skips tiles of D which cannot hold a
 * match according to learned sketches, with every surviving candidate
 * verified exactly (so pruning can lose pairs but never admits a wrong one).
 *
 * The sketch network maps a unit-normalised embedding row x (d values) to a
 * unit 64-d sketch: s = z/|z|, z = W2 GELU(W1 x + b1) + b2 (GELU exact, with
 * the normal CDF).  Parameters are one flat FP32 array, in this order:
 * W1 [hidden x d] row-major, b1 [hidden], W2 [64 x hidden] row-major, b2 [64].
 * Training minimises sum_k w_k (s_pk . s_qk - t_k)^2 / sum_k w_k over labelled
 * pairs (t_k: the pair's exact cosine) with Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8), on the GPU.
 * ------------------------------------------------------------------------- */
typedef struct ejoin_sketch ejoin_sketch;

/* out must be 64.  Parameters start at zero: set them with ejoin_sketch_set_params. */
ejoin_status ejoin_sketch_create(ejoin_ctx *ctx, int32_t d, int32_t hidden, int32_t out, ejoin_sketch **sk);
/* Release the network (synchronises its device; does not use the context, so it may come after ejoin_destroy). */
void ejoin_sketch_destroy(ejoin_sketch *sk);
int64_t ejoin_sketch_num_params(const ejoin_sketch *sk);
/* Host arrays of ejoin_sketch_num_params floats; set also resets the Adam state. */
ejoin_status ejoin_sketch_set_params(ejoin_sketch *sk, const float *h_params);
ejoin_status ejoin_sketch_get_params(const ejoin_sketch *sk, float *h_params);
/* Sketches of the rows of X (device, raw rows; normalised internally) into d_S [X.n x 64]. */
ejoin_status ejoin_sketch_forward(ejoin_sketch *sk, ejoin_rel X, float *d_S);
/* The same on the tensor cores, as the pruned join computes its sketches: both layers are TF32 products
 * of the FP32 operands with FP32 accumulation (bias, GELU and the row scale in the epilogue), so each
 * sketch carries a relative error of about 1e-3 against ejoin_sketch_forward.  Needs X.ld, d and hidden
 * multiples of 4 and a 16-byte aligned X.x (else EJOIN_EUNSUPPORTED). */
ejoin_status ejoin_sketch_forward_tc(ejoin_sketch *sk, ejoin_rel X, float *d_S);
/* Pairs k = (rows d_p[k], d_q[k] of X), d_inv = 1/|row| of X's rows (device, see
 * ejoin_row_inv_norm).  grad: loss and its gradient (flat parameter layout,
 * device, optional) without changing the parameters; train_step: the same
 * followed by one Adam step with learning rate lr.  *h_loss (optional, host)
 * receives the loss (synchronises). */
ejoin_status ejoin_sketch_grad(ejoin_sketch *sk, ejoin_rel X, const float *d_inv, const uint32_t *d_p,
                               const uint32_t *d_q, const float *d_t, const float *d_w, int64_t n_pairs,
                               float *d_grad, float *h_loss);
ejoin_status ejoin_sketch_train_step(ejoin_sketch *sk, ejoin_rel X, const float *d_inv, const uint32_t *d_p,
                                     const uint32_t *d_q, const float *d_t, const float *d_w, int64_t n_pairs,
                                     float lr, float *h_loss);
/* Sketch cosine s_p . s_q of each pair into d_out (device). */
ejoin_status ejoin_sketch_pair_sims(ejoin_sketch *sk, ejoin_rel X, const float *d_inv, const uint32_t *d_p,
                                    const uint32_t *d_q, int64_t n_pairs, float *d_out);
/* 1/|row| of every row of X (FP32, 0 for a zero row) into d_inv. */
ejoin_status ejoin_row_inv_norm(ejoin_ctx *ctx, ejoin_rel X, float *d_inv);
/* Exact FP32 cosine similarity (Sec. III-A) of the pairs (R row d_i[k], S row d_j[k]) into d_sim. */
ejoin_status ejoin_score_pairs(ejoin_ctx *ctx, ejoin_rel R, ejoin_rel S, const uint32_t *d_i, const uint32_t *d_j,
                               int64_t n_pairs, float *d_sim);

/* Training of the sketch network on the GPU, with its labelled set and its calibration.  X_train and
 * X_cal are two held-out device samples of the rows the pruned join will see (raw FP32 rows, at least two
 * each).  Steps, all in the library's kernels:
 *   1. labels: the exact self-join of X_train at eps - label_margin (ejoin_threshold; matches and near
 *      misses, each with its exact FP32 similarity as target, weight w_join), of which a seeded draw keeps
 *      about n_pairs / 2 pairs (i != j), then uniform random row pairs of X_train scored exactly (weight 1)
 *      up to n_pairs in all;
 *   2. epochs: Adam steps (ejoin_sketch_train_step) over batches of the labelled pairs, each epoch in a
 *      seeded order (a keyed bijection of the pair indices);
 *   3. calibration: eps_sketch = the (1 - recall) quantile (linear interpolation between order statistics)
 *      of the sketch cosine over the exact matches of X_cal at eps, less cal_margin.
 * Every draw depends on cfg->seed only.  With init nonzero the parameters are first set to a seeded
 * scaled Gaussian (W1 ~ N(0, 1/d), W2 ~ N(0, 1/hidden), biases 0) and the Adam state is reset; otherwise
 * training continues from the current parameters.  *eps_sketch receives the calibrated threshold for
 * ejoin_threshold_pruned (-1 when X_cal has no match), report (optional) the figures below.  Uses the
 * context's stream and workspace (its statistics then describe the calibration join) and allocates its
 * temporaries; synchronises.  The paper has no learned component. */
typedef struct ejoin_sketch_train_cfg {
    float eps;            /* the join threshold the sketch will prune for */
    float label_margin;   /* labelling join at eps - label_margin (<= 0: 0.2) */
    float w_join;         /* weight of the pairs from the labelling join (<= 0: 8) */
    int64_t n_pairs;      /* labelled pairs (<= 0: 10,000,000; at most 2^31) */
    int32_t epochs;       /* passes over the labelled pairs (<= 0: 3) */
    int32_t batch;        /* pairs per Adam step (<= 0: 65,536) */
    float lr;             /* Adam learning rate (<= 0: 0.002) */
    float recall;         /* target recall of the calibration, in (0, 1] (else 0.999) */
    float cal_margin;     /* subtracted from the calibrated quantile (< 0: 0.01) */
    uint64_t seed;
    int32_t init;         /* nonzero: seeded initialisation of the parameters first */
} ejoin_sketch_train_cfg;

typedef struct ejoin_sketch_train_report {
    uint64_t label_join_pairs;     /* pairs of the labelling join, (i, i) included */
    uint64_t labelled_join;        /* labelled pairs drawn from it */
    uint64_t labelled_random;      /* random labelled pairs */
    float loss_first, loss_last;   /* weighted loss of the first and of the last Adam step's batch */
    uint64_t calibration_matches;  /* exact matches of X_cal at eps */
    float eps_sketch;
    float ms_label, ms_train, ms_calibrate;
} ejoin_sketch_train_report;

ejoin_status ejoin_sketch_train(ejoin_sketch *sk, ejoin_rel X_train, ejoin_rel X_cal,
                                const ejoin_sketch_train_cfg *cfg, float *eps_sketch,
                                ejoin_sketch_train_report *report);

typedef struct ejoin_prune_stats {
    uint64_t tiles_total;  /* 128 x 256 tile pairs of the full join */
    uint64_t tiles_kept;   /* tile pairs whose sketch bound reaches eps_sketch */
    uint64_t candidates, pairs;
    float ms_prepare;      /* normalise + sketch + reorder */
    float ms_bound;        /* tile statistics + tile-pair bounds */
    float ms_contract, ms_rescore, ms_total;
    /* diagnostics of the tile bounds (filled when stats is given): mean angular radius (rad) of the
       used balls of the R tiles (a) and of the S tiles (b), the fraction of used balls wider than
       0.5 rad, the covering anchors of R and the rows of the largest anchor group of R */
    float ball_radius_mean_a, ball_radius_mean_b;
    float wide_ball_frac_a, wide_ball_frac_b;
    uint64_t anchors_a, max_group_rows_a;
    /* the part of ms_prepare spent on R: normalisation and sketches, covering anchors, and anchor
       assignment with the reorder and gathers */
    float ms_sketch_a, ms_cover_a, ms_assign_a;
    /* recall estimate (filled when recall_est is given): the share of the exact matches of the sampled R
       rows that the pruned join returns, the rows sampled and their exact matches */
    float recall_est;
    uint64_t recall_sample_rows, recall_sample_matches;
    float ms_tile_stats;   /* the part of ms_bound spent on the balls of the tiles (the rest: tile-pair bounds) */
    int32_t reserved;
} ejoin_prune_stats;

/* Threshold join of R and S (device, no selection) that contracts only the
 * tile pairs whose sketch bound reaches eps_sketch.  Each side is first
 * reordered by nearest covering anchor (anchors drawn in rounds from the rows
 * of a sample that no anchor covers yet at sketch cosine 0.85, so that every
 * group of similar rows gets an anchor of its own) so that tiles are coherent
 * in sketch space; each tile is described by up to 4
 * balls (farthest-point seeds, rows join the nearest seed: unit centroid c
 * and angular radius rho), and a tile pair is kept when some ball pair has
 * cos(max(0, angle(c_a, c_b) - rho_a - rho_b)) >= eps_sketch, an upper bound
 * on the sketch cosine of every row pair the two balls hold.  Every candidate is re-scored exactly, so the result is a subset of
 * ejoin_threshold's (equal up to the pairs whose sketch cosine is below
 * eps_sketch).  ctx must use BF16, e4m3 or TF32; out as for ejoin_threshold;
 * stats optional.  recall_est (optional): the recall of the returned set
 * against the plain join, estimated on up to 2048 evenly spaced rows of R:
 * their exact join with S runs through the plain path, and a match counts as
 * returned iff its tile pair was kept (that is exactly when the pruned join
 * returns it); the estimate costs that sampled join.  Synchronises. */
ejoin_status ejoin_threshold_pruned(ejoin_ctx *ctx, ejoin_sketch *sk, ejoin_rel R, ejoin_rel S, float eps,
                                    float eps_sketch, ejoin_pairs *out, ejoin_prune_stats *stats,
                                    float *recall_est);

/* Bound on every device-side wait of later calls on ctx, in SM clock cycles
 * (0: 2^31, about one second), as ejoin_config.timeout_cycles.  A wait that
 * runs out makes the call return EJOIN_ETIMEOUT with no valid result; its
 * kernel first lets the copies and MMAs it has issued complete (a fixed bound
 * of its own, about 8 s), frees its tensor memory and returns, so the context
 * stays usable.  No counterpart in the paper (failure detection of the GPU
 * path). */
ejoin_status ejoin_set_timeout(ejoin_ctx *ctx, uint64_t timeout_cycles);

/* Statistics of the last call on ctx. */
ejoin_status ejoin_last_stats(const ejoin_ctx *ctx, ejoin_stats *out);

/* Static text for a status code. */
const char *ejoin_strerror(ejoin_status s);

/* Library version string. */
const char *ejoin_version(void);

/* ---------------------------------------------------------------------------
 * Allocation-free variant of ejoin_threshold.  The paper has no counterpart.
 *
 * For callers that cannot call cudaMalloc: a database executor or serving
 * process whose device memory belongs to its own pool allocator, a process
 * held to a fixed memory budget, or a latency-critical loop in which
 * cudaMalloc / cudaFree would synchronise the device or fail under
 * fragmentation.  It runs the BF16 path (normalise, tcgen05 contraction with
 * the fused threshold, exact re-score) with every piece of scratch in one
 * fixed-size array that lives in the library's device image, and calls no
 * allocating routine.  No selection predicate; no context.
 *
 * R.x, S.x and d_pairs are device pointers on the CURRENT device; the work is
 * enqueued on `stream` (cudaStream_t; NULL = legacy default stream) and the
 * call synchronises that stream before returning.  *count receives the number
 * of result pairs; EJOIN_EOVERFLOW with *count > capacity means the first
 * `capacity` records are valid (as for ejoin_threshold); EJOIN_EOVERFLOW with
 * *count == 0 means the candidates exceeded EJOIN_STATIC_MAX_CANDIDATES and
 * the result is incomplete (use ejoin_threshold for such joins).
 *
 * Limits (EJOIN_EINVAL beyond them): R.n, S.n <= EJOIN_STATIC_MAX_ROWS and
 * (ceil(R.n/256) + ceil(S.n/256)) * 256 * ceil(d/64) * 64 <=
 * EJOIN_STATIC_MAX_OPERAND_ELEMS.  Every GPU that loads the library holds the
 * EJOIN_STATIC_SCRATCH_BYTES array until the process exits.  Every call looks
 * up the array's device address (cudaGetSymbolAddress) with the current device
 * and reads the counts back, synchronising `stream`: do not call it while that
 * stream is being captured into a CUDA graph.  All calls share the array and
 * it keeps the last call's contents; counters are cleared at the start of each
 * call, and calls that overlap on the GPU race on the array.
 * ------------------------------------------------------------------------- */
#define EJOIN_STATIC_MAX_ROWS 65536
#define EJOIN_STATIC_MAX_OPERAND_ELEMS (1u << 24)
#define EJOIN_STATIC_MAX_CANDIDATES (1u << 20)
#define EJOIN_STATIC_SCRATCH_BYTES \
    (1024u + 2u * 4u * EJOIN_STATIC_MAX_ROWS + 2u * 8u * EJOIN_STATIC_MAX_CANDIDATES + 2u * EJOIN_STATIC_MAX_OPERAND_ELEMS)
ejoin_status ejoin_threshold_static(ejoin_rel R, ejoin_rel S, float eps, ejoin_pair *d_pairs, uint64_t capacity,
                                    uint64_t *count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* EJOIN_H */
