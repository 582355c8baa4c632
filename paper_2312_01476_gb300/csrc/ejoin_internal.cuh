// Internal declarations shared by the CUDA translation units of libejoin.
// Device-side PTX wrappers for mbarrier / TMA / tcgen05 (sm_103a), the
// device error word, and the kernel launchers called by the C ABI layer.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ejoin.h"

namespace ej {

// Bits of the device error word (DevMisc::status).
// ERR_RANGE: a row's FP32 sum of squares overflowed or underflowed in a kernel that does not rescale
// (the host repeats the work through the rescaling normalisation pass)
enum : unsigned { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u, ERR_INTERNAL = 4u, ERR_RANGE = 8u };

// Storage format of normalised rows.
enum Fmt : int { FMT_F32 = 0, FMT_BF16 = 1, FMT_FP8 = 2 };

// Device-resident counters of one call (one 64-byte block of the workspace).
struct DevMisc {
    unsigned long long cand_count;  // candidates found by the contraction (may exceed capacity)
    unsigned long long pair_count;  // result pairs written by the re-score (may exceed capacity)
    unsigned long long band_count;  // candidates re-scored in FP64
    long long n_sel[2];             // rows kept by the selection of R (0) and S (1)
    unsigned status;                // ERR_* bits
    unsigned pad;
    unsigned long long pad2[2];
};

struct SelArgs {
    const int32_t *attr;
    int op;
    int c;
    const uint32_t *bits;
};

// Row r passes `attr[r] op c` (when attr is set) and bit r of bits (when bits is set).
__device__ __forceinline__ bool sel_keep(const SelArgs &s, int64_t r)
{
    bool k = true;
    if (s.attr) {
        const int a = s.attr[r];
        switch (s.op) {
        case EJOIN_LT: k = a < s.c; break;
        case EJOIN_LE: k = a <= s.c; break;
        case EJOIN_GT: k = a > s.c; break;
        case EJOIN_GE: k = a >= s.c; break;
        case EJOIN_EQ: k = a == s.c; break;
        case EJOIN_NE: k = a != s.c; break;
        default: k = false;
        }
    }
    if (k && s.bits) k = (s.bits[r >> 5] >> (r & 31)) & 1u;
    return k;
}

// Job table of a batched contraction (device arrays).  Job j owns the tiles
// [tile_off[j], tile_off[j+1]) of the global tile space, the operand rows
// [a_off[j], a_off[j] + nA[j]) of the concatenated R operand and
// [b_off[j], b_off[j] + nB[j]) of the concatenated S operand, and compares
// against thr[j].
struct BatchTables {
    const long long *tile_off;
    const long long *a_off;
    const long long *b_off;
    const int *nA;
    const int *nB;
    const float *thr;
    int n_jobs;
    // tile-list mode (pruned joins): the tiles to run are tile_list[0 .. min(*tile_count, tile_cap))
    const uint2 *tile_list;
    const unsigned long long *tile_count;
    unsigned long long tile_cap;
    // tile-list mode of a self-join listing only block pairs on and above the diagonal of 256-row
    // blocks: inside a diagonal block (row tile m, column tile n, m / 2 == n) keep col >= row
    int sym;
    // top-k passes.  Pass 0: row_best[r * top_ld + (c >> top_shift)] = the largest bulk similarity
    // (order-preserving bits, f2ord) of operand row r of A over the column group of c (one group for
    // top-1).  Pass 1: row_best[r] = a lower bound of row r's k-th largest bulk similarity, and the
    // margin below it that the candidate pass keeps
    unsigned *row_best;
    long long top_ld;
    int top_shift;
    // pass 0 may sample every top_stride-th column tile while that leaves at least top_min_tiles
    int top_stride, top_min_tiles;
    float top_margin;
    // GEMM mode (a dense layer): out[r * out_ld + c] = act(rowscale[r] * acc(r, c) + bias[c]) for the valid
    // rows and columns; rowscale and bias optional, act: 0 none, 1 exact GELU
    const float *g_rowscale;
    const float *g_bias;
    float *g_out;
    long long g_ld;
    int g_act;
};

// Order-preserving map of floats to unsigned integers (and back): a < b iff f2ord(a) < f2ord(b)
// for non-NaN a, b; 0 lies below the image of every float.
__host__ __device__ __forceinline__ unsigned f2ord(float f)
{
#if defined(__CUDA_ARCH__)
    const unsigned u = __float_as_uint(f);
#else
    unsigned u;
    __builtin_memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ __forceinline__ float ord2f(unsigned o)
{
    const unsigned u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float f;
    __builtin_memcpy(&f, &u, 4);
    return f;
#endif
}

// Per-job row sources of a batched re-score (device arrays).  Operand row a of job j is row
// idsA[a] - srcA_off[j] of R_j when the batch has selections (idsA: the kept rows' indices among all of
// the jobs' concatenated rows, srcA_off: the jobs' offsets there), else row a - a_off[j]; likewise for S.
struct BatchRows {
    const float *const *R;
    const long long *ldR;
    const float *const *S;
    const long long *ldS;
    const long long *a_off;
    const long long *b_off;
    const float *eps;
    int n_jobs;
    const uint32_t *idsA = nullptr, *idsB = nullptr;
    const long long *srcA_off = nullptr, *srcB_off = nullptr;
};

// Original row of operand row a of job j (see BatchRows).
__device__ __forceinline__ uint32_t batch_row_a(const BatchRows &br, uint32_t a, uint32_t j)
{
    return br.idsA ? (uint32_t)((long long)__ldg(br.idsA + a) - __ldg(br.srcA_off + j))
                   : (uint32_t)((long long)a - __ldg(br.a_off + j));
}
__device__ __forceinline__ uint32_t batch_row_b(const BatchRows &br, uint32_t b, uint32_t j)
{
    return br.idsB ? (uint32_t)((long long)__ldg(br.idsB + b) - __ldg(br.srcB_off + j))
                   : (uint32_t)((long long)b - __ldg(br.b_off + j));
}

// Arguments of the re-score fused into the contraction (single join).
struct FuseArgs {
    const float *R;
    int64_t ldR;
    const float *S;
    int64_t ldS;
    int d;
    const uint32_t *idsR, *idsS;
    const float *invR, *invS;
    float eps, fp64_band;
    ejoin_pair *out;
    uint64_t out_cap;
    unsigned long long *pair_count, *band_count;
    int count_only;
};

// One result record of a batched join.
struct BatchPair {
    uint32_t job, i, j;
    float sim;
};

// Rows per selection block (count / scatter kernels).
constexpr int SEL_THREADS = 512;
constexpr int SEL_ITEMS = 16;
constexpr int64_t SEL_ROWS_PER_BLOCK = (int64_t)SEL_THREADS * SEL_ITEMS;

// ---------------------------------------------------------------- launchers
cudaError_t launch_sel_count(const SelArgs &s, int64_t n, uint32_t *block_counts, cudaStream_t st);
cudaError_t launch_sel_scan(const uint32_t *block_counts, int64_t n_blocks, uint32_t *block_offsets,
                            long long *n_sel, cudaStream_t st);
cudaError_t launch_sel_scatter(const SelArgs &s, int64_t n, const uint32_t *block_offsets, uint32_t *ids,
                               cudaStream_t st);
cudaError_t launch_set_count(long long *n_sel, long long value, cudaStream_t st);
// raw_out (optional): each normalised row's FP32 values are also copied to raw_out + r * raw_ld, r its
// source row number (a device copy of rows read from host memory).
cudaError_t launch_normalize(int fmt, const float *x, int64_t ld, int d, const uint32_t *ids,
                             const long long *n_rows_dev, int64_t n_rows_max, void *out, int64_t ld_out,
                             int kp, float *inv_norm, float *scale, unsigned *status, int num_sms,
                             cudaStream_t st, float *raw_out = nullptr, int64_t raw_ld = 0);
// e4m3 normalisation whose scales are shared by each aligned group of `group` output rows
// (scale[c] = the largest per-row scale of c's group); 3 kernels.
cudaError_t launch_normalize_fp8_grouped(const float *x, int64_t ld, int d, const uint32_t *ids,
                                         const long long *n_rows_dev, int64_t n_rows_max, void *out, int64_t ld_out,
                                         int kp, float *inv_norm, float *scale, int group, unsigned *status,
                                         int num_sms, cudaStream_t st, float *raw_out = nullptr,
                                         int64_t raw_ld = 0);
cudaError_t launch_normalize_batch(int fmt, const float *const *xs, const long long *lds, const long long *row_off,
                                   int n_rel, int64_t total_rows, int d, void *out, int kp, float *inv_norm,
                                   float *scale, unsigned *status, int num_sms, cudaStream_t st,
                                   bool aligned = false,
                                   const uint32_t *ids = nullptr, const long long *src_off = nullptr);
cudaError_t launch_sim_simt(const float *A, const float *B, int kp, const long long *nA, const long long *nB,
                            float thr, uint2 *cand, uint64_t cap, unsigned long long *cand_count,
                            int count_only, int num_sms, cudaStream_t st);
// kind: 0 = BF16 (kind::f16), 1 = e4m3 (kind::f8f6f4), 2 = TF32 (kind::tf32)
cudaError_t launch_sim_tc(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp,
                          const long long *nA, const long long *nB, float thr, const float *scaleA,
                          const float *scaleB, uint2 *cand, uint64_t cap, unsigned long long *cand_count,
                          unsigned *status, uint64_t timeout, int count_only, int grid, int group_m,
                          cudaStream_t st);
// Self-join contraction (one operand, nA rows): only the block pairs on and above the
// diagonal of 256-row blocks; candidates (r, c) have r <= c.
cudaError_t launch_sim_tc_sym(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                              float thr, const float *scale, uint2 *cand, uint64_t cap,
                              unsigned long long *cand_count, unsigned *status, uint64_t timeout, int count_only,
                              int grid, int group_m, cudaStream_t st);
// Top-k passes of the contraction (single join): pass 0 records in row_best[r * top_ld + (c >> top_shift)]
// the largest bulk similarity of operand row r of A over the column group of c (atomicMax on f2ord;
// row_best zeroed by the caller; top_shift >= 7, the 128 columns of an epilogue lane stay in one group),
// over every top_stride-th 256-column tile only while at least top_min_tiles tiles remain (groups
// without a sampled tile stay 0);
// pass 1 emits the candidates (r, c) with bulk similarity >= ord2f(row_best[r]) - margin; pass 2 is
// top-1 in one pass: per tile, row_best[r] is raised to the row's tile maximum and the columns
// within margin of the raised value are emitted (row_best zeroed by the caller).
cudaError_t launch_sim_tc_top(int kind, int pass, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp,
                              const long long *nA, const long long *nB, const float *scaleA, const float *scaleB,
                              unsigned *row_best, long long top_ld, int top_shift, int top_stride, int top_min_tiles,
                              float margin, uint2 *cand, uint64_t cap, unsigned long long *cand_count,
                              unsigned *status, uint64_t timeout, int grid, int group_m, cudaStream_t st);
// Contraction with the exact re-score fused in (extra warps consume the candidates from a
// shared-memory ring and write final pairs).  Needs 16-byte aligned rows, ld % 4 == 0 and
// d % 4 == 0.
cudaError_t launch_sim_tc_fused(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp,
                                const long long *nA, const long long *nB, float thr, const float *scaleA,
                                const float *scaleB, const FuseArgs &fa, unsigned long long *cand_count,
                                unsigned *status, uint64_t timeout, int grid, int group_m, cudaStream_t st);
// Dense layer on the tensor cores (TF32 from FP32 operands, FP32 accumulation): out = act(rowscale * A B^T + bias)
// for A [nA x kp] and B [nB x kp] (tensor maps as for the contraction, kind TF32), out [nA x nB] with row
// stride out_ld; act 0 none, 1 exact GELU.
cudaError_t launch_gemm_tc(const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                           const long long *nB, const float *rowscale, const float *bias, int act, float *out,
                           long long out_ld, unsigned *status, uint64_t timeout, int grid, cudaStream_t st);
// Contraction over an explicit list of (row tile, column tile) pairs (pruned joins); sym: see
// BatchTables::sym.
cudaError_t launch_sim_tc_list(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                               const long long *nB, float thr, const uint2 *tile_list,
                               const unsigned long long *tile_count, unsigned long long tile_cap, uint2 *cand,
                               uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout,
                               int grid, cudaStream_t st, int sym = 0);
// Batched contraction over a job table (BF16 / e4m3 / TF32 kinds as above).
cudaError_t launch_sim_tc_batch(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp,
                                const BatchTables &bt, const float *scaleA, const float *scaleB, uint2 *cand,
                                uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout,
                                int grid, int group_m, cudaStream_t st);
cudaError_t launch_score_pairs(const float *R, int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *pi,
                               const uint32_t *pj, const float *invR, const float *invS, int64_t n, float *out,
                               int num_sms, cudaStream_t st);
// Streaming batched re-score (16-byte aligned rows, d % 4 == 0, d <= 1024): candidates counting-sorted into
// `sorted` (cand_cap entries) by job, S block of sblock_rows rows within the job and A row, then re-scored by
// warps that keep the A row in registers and the S rows in flight through a shared-memory ring; records and
// counts identical to launch_rescore_batch.  bbase[j]: first bucket of job j (n_jobs + 1 entries, the last
// n_buckets), nA[j]: its A rows.  buf: rescore_stream_batch_buf_bytes(n_buckets, rows_a) bytes.
size_t rescore_stream_batch_buf_bytes(int64_t n_buckets, int64_t rows_a);
cudaError_t launch_rescore_stream_batch(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                        uint2 *sorted, void *buf, int64_t rows_a, const BatchRows &br,
                                        const long long *bbase, const int *nA, int64_t n_buckets, int64_t sblock_rows,
                                        int d, const float *invA, const float *invB, float fp64_band, BatchPair *out,
                                        uint64_t out_cap, unsigned long long *out_count,
                                        unsigned long long *band_count, int num_sms, cudaStream_t st);
cudaError_t launch_rescore_batch(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                 const BatchRows &br, int d, const float *invA, const float *invB, float fp64_band,
                                 BatchPair *out, uint64_t out_cap, unsigned long long *out_count,
                                 unsigned long long *band_count, bool aligned, int num_sms, cudaStream_t st);
// Default row-tile group width of the contraction's raster for operands of
// padded dimension kp: about 40 MB of FP32 input rows per group (the R rows the
// re-score gathers while the group's candidates are processed stay in L2).
inline int default_group_m(int64_t kp)
{
    int64_t g = (40ll << 20) / (128 * 4 * (kp > 0 ? kp : 1));
    if (g < 8) g = 8;
    if (g > 256) g = 256;
    return (int)g;
}
size_t sim_tc_smem_bytes();
// ℰ-selection scan (esel.cu): candidates (row of R, col_base + c) for the queries c < m with
// acc >= thr_rel * ||row||, acc the TF32 product of the FP32 rows (tmR: box 32 x 128, 128-byte swizzle)
// with up to 64 normalised queries (tmQ: box 32 x 64); writes 1/||row|| to inv_out when given.
// nR: device row count.  ERR_RANGE in *status: a row's sum of squares left the FP32 range.
cudaError_t launch_esel(const CUtensorMap *tmR, const CUtensorMap *tmQ, int num_kb, const long long *nR, int m,
                        int col_base, float thr_rel, float *inv_out, uint2 *cand, uint64_t cap,
                        unsigned long long *cand_count, unsigned *status, uint64_t timeout, int grid, cudaStream_t st);
// Top-k join condition (topk.cu).  Group maxima per row of the first pass: at most this many.
constexpr int64_t TOPK_MAX_GROUPS = 8192;
constexpr int TOPK_MAX_K = 32;
constexpr int TOPK_SAMPLE_STRIDE = 8;  // column-tile stride of the first top-k pass
// Every candidate's similarity is the FP32 cosine from the raw rows, as the threshold re-score's.
// k = 1: best[r] = max over the candidates (r, c) of (f2ord(sim) << 32 | ~original j) (best zeroed
// by the caller); then out[r] = (i, j, sim) for every operand row r of A (rows without a best are
// counted in *missing).
cudaError_t launch_top1_rescore(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                const float *R, int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *idsR,
                                const uint32_t *idsS, const float *invR, const float *invS, unsigned long long *best,
                                int num_sms, cudaStream_t st);
cudaError_t launch_top1_emit(const unsigned long long *best, const long long *nA_dev, int64_t nA_max,
                             const uint32_t *idsR, ejoin_pair *out, uint64_t out_cap, unsigned long long *missing,
                             int num_sms, cudaStream_t st);
// k > 1: thr[r] = the k-th largest of row r's group maxima gmax[r * ld + g], g < ceil(nB / 2^shift)
// (f2ord(-inf) when there are fewer than k groups), a lower bound of its k-th largest bulk similarity.
cudaError_t launch_topk_threshold(const unsigned *gmax, int64_t ld, int shift, const long long *nA_dev,
                                  int64_t nA_max, const long long *nB_dev, int k, unsigned *thr, int num_sms,
                                  cudaStream_t st);
// keys[t] = f2ord(sim) << 32 | ~original j of candidate t, and row_cnt[r] += candidates of row r.
cudaError_t launch_topk_rescore(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                const float *R, int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *idsR,
                                const uint32_t *idsS, const float *invR, const float *invS, unsigned long long *keys,
                                unsigned *row_cnt, int num_sms, cudaStream_t st);
// seg[row_off[r] + t] = the keys of row r's candidates (row_fill zeroed by the caller).
cudaError_t launch_topk_scatter(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                const unsigned long long *keys, const unsigned *row_off, unsigned *row_fill,
                                unsigned long long *seg, int num_sms, cudaStream_t st);
// out[r * kk + t] = row r's (t+1)-th largest key as (i, j, sim), t < kk (a row with fewer than kk keys
// is counted in *missing and padded with (i, ~0u, -inf)).
cudaError_t launch_topk_select(const unsigned long long *seg, const unsigned *row_off, const unsigned *row_cnt,
                               const long long *nA_dev, int64_t nA_max, int kk, const uint32_t *idsR, ejoin_pair *out,
                               uint64_t out_cap, unsigned long long *missing, int num_sms, cudaStream_t st);
// Workspace of the accurate tier's squared row norms (compensated dot products finished in FP64): per
// row of R (nR rows) and of S (nS rows) a claim word and a norm.  When a launcher gets one, the rows listed in
// the band list have their norms computed once, and each listed candidate only its cross product; the
// similarities are the same bit for bit.
struct BandNorms {
    unsigned *claimR = nullptr, *claimS = nullptr;  // contiguous: claimS = claimR + nR
    double *nrmR = nullptr, *nrmS = nullptr;
    int64_t nR = 0, nS = 0;
};

// Candidates: cand[0 .. min(*cand_count, cand_cap)).  Candidates whose FP32 similarity
// lies within fp64_band of eps are listed in band_list (capacity band_cap >= cand_cap,
// counted in *band_count) and decided by a second kernel, the accurate tier.  mirror: the
// candidates come from the upper triangle of a self-join; each pair (i, j), i != j, is
// written in both orders.
cudaError_t launch_rescore(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                           const float *R, int64_t ldR, const float *S, int64_t ldS, int d,
                           const uint32_t *idsR, const uint32_t *idsS, const float *invR, const float *invS,
                           float eps, float fp64_band, ejoin_pair *out, uint64_t out_cap,
                           unsigned long long *out_count, unsigned long long *band_count, int count_only,
                           int num_sms, cudaStream_t st, uint2 *band_list, uint64_t band_cap, int mirror = 0,
                           const BandNorms *bn = nullptr);

// Panel-ordered re-score (same decisions and similarities as launch_rescore, bit for bit): the candidates
// are bucketed into `sorted` (cand_cap entries) by (block of S rows sized for L2, panel of
// rescore_panel_rows(d) consecutive operand rows of R), and each panel's FP32 R rows are staged in shared
// memory once, so only the S rows are gathered per candidate.  Needs d % 4 == 0, d <= 1024,
// ldR % 4 == 0, ldS % 4 == 0 and 16-byte aligned R and S (cudaErrorInvalidValue otherwise); panel_buf
// holds rescore_panel_buf_bytes(n_rows, n_rows_s, d, cand_hint) bytes, n_rows and n_rows_s upper bounds of
// the operand rows of R (*nA_dev at run time) and of S, cand_hint the number of candidates (0: unknown;
// S blocks then split the panels by the L2 size only).
int rescore_panel_rows(int d);
size_t rescore_panel_buf_bytes(int64_t n_rows, int64_t n_rows_s, int d, uint64_t cand_hint);
cudaError_t launch_rescore_panels(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                  uint2 *sorted, void *panel_buf, int64_t n_rows, int64_t n_rows_s,
                                  uint64_t cand_hint, const long long *nA_dev, const float *R, int64_t ldR, const float *S, int64_t ldS,
                                  int d, const uint32_t *idsR, const uint32_t *idsS, const float *invR,
                                  const float *invS, float eps, float fp64_band, ejoin_pair *out, uint64_t out_cap,
                                  unsigned long long *out_count, unsigned long long *band_count, int count_only,
                                  int num_sms, cudaStream_t st, uint2 *band_list, uint64_t band_cap, int mirror,
                                  const BandNorms *bn = nullptr);

// Sort of n result records by (i, j) ascending (sort.cu), i < n_i and j < n_j: LSD radix sort over the
// significant bits of j, then of i, ping-ponging between data and tmp (n records); the result ends in
// data.  scratch holds sort_pairs_scratch_bytes(n) bytes; n < 2^32.
size_t sort_pairs_scratch_bytes(uint64_t n);
cudaError_t launch_sort_pairs(ejoin_pair *data, ejoin_pair *tmp, uint64_t n, uint64_t n_i, uint64_t n_j,
                              void *scratch, cudaStream_t st);

// ------------------------------------------------------- device PTX helpers
#if defined(__CUDACC__)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  Gives up (returns false) after
// `timeout` SM cycles or when another role has raised the CTA's abort flag;
// the first role to time out raises the flag and the device error word.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t timeout,
                                                  volatile int *abort_flag, unsigned *status)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((uint64_t)(clock64() - t0) > timeout) {
            *abort_flag = 1;
            atomicOr(status, ERR_TIMEOUT);
            return false;
        }
    }
}

// Wait for asynchronous work this CTA has already issued (TMA copies landing in its shared memory, MMAs
// writing its TMEM) before it frees TMEM or exits.  Issued copies and MMAs always complete, in
// microseconds, so this wait does not use the caller's timeout, which may be set short enough to expire
// while they are in flight: it has a fixed bound of its own (DRAIN_CYCLES, about 8 s at 2 GHz), after
// which it records ERR_TIMEOUT and returns.
constexpr uint64_t DRAIN_CYCLES = 1ull << 34;
__device__ __forceinline__ void mbar_drain_wait(uint32_t bar, uint32_t parity, unsigned *status)
{
    if (mbar_try_wait(bar, parity)) return;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if ((uint64_t)(clock64() - t0) > DRAIN_CYCLES) {
            atomicOr(status, ERR_TIMEOUT);
            return;
        }
    }
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// 2-D tiled TMA load of one box into shared memory; completion is signalled
// on `bar` as transaction bytes.  x = innermost (element) coordinate.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t holder_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(holder_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Arrive on `bar` once every tcgen05 operation issued so far by this thread completes.
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile written by TMA
// with 128-byte swizzling: rows of 128 bytes, 8-row core groups 1024 bytes
// apart (stride byte offset), leading byte offset unused for this layout,
// descriptor version 1, layout type 2 = SWIZZLE_128B.  The tile base must be
// 1024-byte aligned; advancing along K inside the 128-byte row is done by
// adding the byte offset to the start address.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Wait for outstanding tcgen05.ld and tie the wait to the destination
// registers, so that no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&v)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]),
                   "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]),
                   "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}

// ---------------------------------------------------- compensated dot products
// The accurate tier of the re-score: x.y, x.x and y.y of two FP32 rows with the
// compensated dot product "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci.
// Comput. 26(6), 2005): every product is split exactly into p + e with one
// FMA, every running sum into s + t with the branch-free two-sum, and the
// error terms are summed alongside.  The result carries the accuracy of an
// evaluation in twice the working precision, |err| <= u |dot| + gamma_n^2
// sum |x_k y_k| (u = 2^-24, gamma_n = n u / (1 - n u)); here the high and low
// parts are added in FP64, so the u |dot| rounding term is not incurred.  For
// d = 768 the relative error is below 3e-9 of |x| |y|, and on GB300 it costs a
// fraction of a plain FP64 dot product.  The lanes of a warp each take the
// elements k = lane, lane + 32, ...; partial (sum, error) pairs are combined
// with the same two-sum.
struct Dot2Acc {
    float s, c;  // running sum and accumulated error
};

// (the _rn intrinsics keep the compiler from contracting or reassociating these steps)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void dot2_add(Dot2Acc &a, float x, float y)
{
    const float p = __fmul_rn(x, y);
    const float ep = fmaf(x, y, -p);  // exact: x y = p + ep
    float s, es;
    two_sum(a.s, p, s, es);
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(es, ep));
}

__device__ __forceinline__ double dot2_warp_total(Dot2Acc a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, a.s, o);
        const float oc = __shfl_xor_sync(0xffffffffu, a.c, o);
        float s, e;
        two_sum(a.s, os, s, e);
        a.s = s;
        a.c = __fadd_rn(a.c, __fadd_rn(oc, e));
    }
    return (double)a.s + (double)a.c;
}

// Accurate cosine of two raw FP32 rows (one warp): Dot2 for x.y, x.x, y.y,
// finished in FP64; 0 when a row is zero; clamped to [-1, 1].  Not inlined:
// the callers take it rarely, and its registers must not count against their
// occupancy.
static __device__ __noinline__ double accurate_cosine(const float *__restrict__ r, const float *__restrict__ s, int d,
                                                  int lane)
{
    Dot2Acc xy{0.f, 0.f}, xx{0.f, 0.f}, yy{0.f, 0.f};
    for (int k = lane; k < d; k += 32) {
        const float x = __ldg(r + k), y = __ldg(s + k);
        dot2_add(xy, x, y);
        dot2_add(xx, x, x);
        dot2_add(yy, y, y);
    }
    const double dd = dot2_warp_total(xy), nr = dot2_warp_total(xx), ns = dot2_warp_total(yy);
    double c = (nr > 0.0 && ns > 0.0) ? dd / (sqrt(nr) * sqrt(ns)) : 0.0;
    return fmin(1.0, fmax(-1.0, c));
}

// The same for 16-byte aligned rows with d % 4 == 0: float4 loads, two sets of
// accumulators (even and odd float4 groups of a lane) combined at the end.
static __device__ __noinline__ double accurate_cosine4(const float *__restrict__ r, const float *__restrict__ s, int d,
                                                       int lane)
{
    Dot2Acc xy[2] = {{0.f, 0.f}, {0.f, 0.f}}, xx[2] = {{0.f, 0.f}, {0.f, 0.f}}, yy[2] = {{0.f, 0.f}, {0.f, 0.f}};
    const float4 *r4 = reinterpret_cast<const float4 *>(r), *s4 = reinterpret_cast<const float4 *>(s);
    const int d4 = d >> 2;
    int g = lane;
    for (; g + 32 < d4; g += 64) {
        const float4 a0 = __ldg(r4 + g), b0 = __ldg(s4 + g), a1 = __ldg(r4 + g + 32), b1 = __ldg(s4 + g + 32);
        dot2_add(xy[0], a0.x, b0.x), dot2_add(xy[1], a1.x, b1.x);
        dot2_add(xy[0], a0.y, b0.y), dot2_add(xy[1], a1.y, b1.y);
        dot2_add(xy[0], a0.z, b0.z), dot2_add(xy[1], a1.z, b1.z);
        dot2_add(xy[0], a0.w, b0.w), dot2_add(xy[1], a1.w, b1.w);
        dot2_add(xx[0], a0.x, a0.x), dot2_add(xx[1], a1.x, a1.x);
        dot2_add(xx[0], a0.y, a0.y), dot2_add(xx[1], a1.y, a1.y);
        dot2_add(xx[0], a0.z, a0.z), dot2_add(xx[1], a1.z, a1.z);
        dot2_add(xx[0], a0.w, a0.w), dot2_add(xx[1], a1.w, a1.w);
        dot2_add(yy[0], b0.x, b0.x), dot2_add(yy[1], b1.x, b1.x);
        dot2_add(yy[0], b0.y, b0.y), dot2_add(yy[1], b1.y, b1.y);
        dot2_add(yy[0], b0.z, b0.z), dot2_add(yy[1], b1.z, b1.z);
        dot2_add(yy[0], b0.w, b0.w), dot2_add(yy[1], b1.w, b1.w);
    }
    if (g < d4) {
        const float4 a0 = __ldg(r4 + g), b0 = __ldg(s4 + g);
        dot2_add(xy[0], a0.x, b0.x), dot2_add(xy[0], a0.y, b0.y), dot2_add(xy[0], a0.z, b0.z),
            dot2_add(xy[0], a0.w, b0.w);
        dot2_add(xx[0], a0.x, a0.x), dot2_add(xx[0], a0.y, a0.y), dot2_add(xx[0], a0.z, a0.z),
            dot2_add(xx[0], a0.w, a0.w);
        dot2_add(yy[0], b0.x, b0.x), dot2_add(yy[0], b0.y, b0.y), dot2_add(yy[0], b0.z, b0.z),
            dot2_add(yy[0], b0.w, b0.w);
    }
    // fold the second set into the first (two-sum of the sums, errors added)
    auto fold = [](Dot2Acc &a, const Dot2Acc &b) {
        float t, e;
        two_sum(a.s, b.s, t, e);
        a.s = t;
        a.c = __fadd_rn(a.c, __fadd_rn(b.c, e));
    };
    fold(xy[0], xy[1]);
    fold(xx[0], xx[1]);
    fold(yy[0], yy[1]);
    const double dd = dot2_warp_total(xy[0]), nr = dot2_warp_total(xx[0]), ns = dot2_warp_total(yy[0]);
    double c = (nr > 0.0 && ns > 0.0) ? dd / (sqrt(nr) * sqrt(ns)) : 0.0;
    return fmin(1.0, fmax(-1.0, c));
}

// One compensated dot product x.y of two raw FP32 rows (one warp), finished in FP64, with the lane
// partition and the order of accurate_cosine (plain) or accurate_cosine4 (VEC: 16-byte aligned rows,
// d % 4 == 0).  accurate_dot(r, r) is bit for bit the x.x of accurate_cosine, so squared norms computed
// once per row give that function's value: dd / (sqrt(nr) sqrt(ns)).
template <bool VEC>
static __device__ __noinline__ double accurate_dot(const float *__restrict__ r, const float *__restrict__ s, int d,
                                                   int lane)
{
    if constexpr (!VEC) {
        Dot2Acc xy{0.f, 0.f};
        for (int k = lane; k < d; k += 32) dot2_add(xy, __ldg(r + k), __ldg(s + k));
        return dot2_warp_total(xy);
    } else {
        Dot2Acc xy[2] = {{0.f, 0.f}, {0.f, 0.f}};
        const float4 *r4 = reinterpret_cast<const float4 *>(r), *s4 = reinterpret_cast<const float4 *>(s);
        const int d4 = d >> 2;
        int g = lane;
        for (; g + 32 < d4; g += 64) {
            const float4 a0 = __ldg(r4 + g), b0 = __ldg(s4 + g), a1 = __ldg(r4 + g + 32), b1 = __ldg(s4 + g + 32);
            dot2_add(xy[0], a0.x, b0.x), dot2_add(xy[1], a1.x, b1.x);
            dot2_add(xy[0], a0.y, b0.y), dot2_add(xy[1], a1.y, b1.y);
            dot2_add(xy[0], a0.z, b0.z), dot2_add(xy[1], a1.z, b1.z);
            dot2_add(xy[0], a0.w, b0.w), dot2_add(xy[1], a1.w, b1.w);
        }
        if (g < d4) {
            const float4 a0 = __ldg(r4 + g), b0 = __ldg(s4 + g);
            dot2_add(xy[0], a0.x, b0.x), dot2_add(xy[0], a0.y, b0.y), dot2_add(xy[0], a0.z, b0.z),
                dot2_add(xy[0], a0.w, b0.w);
        }
        float t, e;
        two_sum(xy[0].s, xy[1].s, t, e);
        xy[0].s = t;
        xy[0].c = __fadd_rn(xy[0].c, __fadd_rn(xy[1].c, e));
        return dot2_warp_total(xy[0]);
    }
}

#endif  // __CUDACC__

}  // namespace ej
