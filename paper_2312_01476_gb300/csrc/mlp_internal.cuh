// Internal declarations of the learned-sketch kernels (mlp.cu, prune.cu).
#pragma once

#include <algorithm>

#include "ejoin_internal.cuh"

namespace ej {

enum : int { ACT_NONE = 0, ACT_GELU = 1 };

// C[M x N] = act(rowscale_i * sum_k A(i,k) B(k,j) + bias_j), FP32.
//   A(i,k) = A[r * a_rs + k * a_cs] * (ascale ? ascale[r] : 1), r = aidx ? aidx[i] : i
//   B(k,j) = B[q * b_rs + j * b_cs] * (bscale ? bscale[q] : 1), q = bidx ? bidx[k] : k
// pre (optional) receives the pre-activation.  atomic_acc: split K over CTAs
// and atomically add into a C the caller zeroed (no bias / activation then).
struct GemmArgs {
    const float *A = nullptr;
    const uint32_t *aidx = nullptr;
    const float *ascale = nullptr;
    int64_t a_rs = 0, a_cs = 1;
    const float *B = nullptr;
    const uint32_t *bidx = nullptr;
    const float *bscale = nullptr;
    int64_t b_rs = 0, b_cs = 1;
    float *C = nullptr;
    int64_t ldc = 0;
    const float *bias = nullptr;
    const float *rowscale = nullptr;
    float *pre = nullptr;
    int64_t M = 0, N = 0, K = 0;
    int act = ACT_NONE;
    int atomic_acc = 0;
    int64_t k_chunk = 0;
};

cudaError_t launch_gemm_f32(const GemmArgs &g, int num_sms, cudaStream_t st);
// C = act(rowscale[i] * A W^T + bias) with A (M x K) and W (N x K) contiguous along k (the inference form of a
// layer); needs K % 16 == 0, lda and ldw multiples of 4 and 16-byte aligned A and W (else cudaErrorInvalidValue).
cudaError_t launch_gemm_nt_f32(const float *A, int64_t lda, const float *W, int64_t ldw, const float *bias,
                               const float *rowscale, int act, float *C, int64_t ldc, int64_t M, int N, int K,
                               cudaStream_t st);
cudaError_t launch_rownorm(const float *z, int64_t n, int k, float *s, float *nz, int num_sms, cudaStream_t st);
// wsum: device pointer to the sum of the pair weights.
cudaError_t launch_pair_grad(const float *s, int64_t B, int k, const float *t, const float *w, const float *wsum,
                             float *ds, float *loss, int num_sms, cudaStream_t st);
cudaError_t launch_pair_dot(const float *s, int64_t B, int k, float *out, int num_sms, cudaStream_t st);
cudaError_t launch_row_inv_norm(const float *x, int64_t n, int d, int64_t ld, float *inv, int num_sms, cudaStream_t st);
cudaError_t launch_rownorm_backward(const float *s, const float *ds, const float *nz, int64_t n, int k, float *dz,
                                    int num_sms, cudaStream_t st);
cudaError_t launch_gelu_backward(float *dh, const float *a, int64_t n, int num_sms, cudaStream_t st);
cudaError_t launch_colsum(const float *x, int64_t n, int k, float *out, int num_sms, cudaStream_t st);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, int step, int num_sms, cudaStream_t st);

// ---- training set-up (train.cu); draws are functions of (seed, index) only
// params = [W1 (hid x d) ~ N(0, 1/d), b1 = 0, W2 (out x hid) ~ N(0, 1/hid), b2 = 0]
cudaError_t launch_init_params(float *params, int d, int hid, int out, uint64_t seed, int num_sms, cudaStream_t st);
// The join pairs (i, j), i != j, whose draw falls below keep / 2^32, in input order, as labelled pairs
// (p, q, target = the pair's similarity, weight w_join), the first cap of them written; *d_total = their
// number.  scratch holds label_scratch_bytes(n) bytes (a multiple of 16).
size_t label_scratch_bytes(uint64_t n_join);
cudaError_t launch_label_join_pairs(const ejoin_pair *pairs, uint64_t n, uint64_t seed, uint32_t keep, float w_join,
                                    void *scratch, unsigned long long *d_total, uint64_t cap, uint32_t *p, uint32_t *q,
                                    float *t, float *w, cudaStream_t st);
// n_pairs uniform random row pairs of [0, n_rows)^2 with weight 1 (targets are scored separately).
cudaError_t launch_random_pairs(uint32_t *p, uint32_t *q, float *w, int64_t n_pairs, uint32_t n_rows, uint64_t seed,
                                int num_sms, cudaStream_t st);
// Batch [b0, b0 + m) of epoch `epoch`'s order of the n labelled pairs (a seeded bijection of [0, n)).
cudaError_t launch_gather_batch(const uint32_t *p, const uint32_t *q, const float *t, const float *w, uint64_t n,
                                uint64_t seed, int epoch, uint64_t b0, int64_t m, uint32_t *bp, uint32_t *bq,
                                float *bt, float *bw, int num_sms, cudaStream_t st);
// rec[k] = {f2ord(v[k]), k, v[k]}: sorted by (i, j) they list the values in ascending order.
cudaError_t launch_value_records(const float *v, int64_t n, ejoin_pair *rec, int num_sms, cudaStream_t st);
// Recall probe of a pruned join: *found = the exact matches (i', j) in `pairs` (rows i' * stride of R) whose
// tile pair (position of i in A / 128, position of j in B / 256; either orientation when sym) is in the
// kept list.  permA / permB: position -> original row.  scratch holds recall_probe_scratch_bytes bytes (a
// multiple of 16).
size_t recall_probe_scratch_bytes(int64_t nA, int64_t nB, int64_t tA, int64_t tB);
cudaError_t launch_recall_probe(const uint32_t *permA, int64_t nA, const uint32_t *permB, int64_t nB,
                                const uint2 *list, const unsigned long long *list_count, uint64_t list_cap,
                                int64_t tA, int64_t tB, const ejoin_pair *pairs, uint64_t n_pairs, uint32_t stride,
                                int sym, void *scratch, unsigned long long *found, int num_sms, cudaStream_t st);
// ---- pruning (prune.cu)
// key[r] = base[r] * n_anchor + argmax_a <S[r], anchors[group(r) * n_anchor + a]>, where group(r) =
// grp ? grp[r] : 0 (anchors of group g are rows g * n_anchor .. of `anchors`).
cudaError_t launch_assign_keys(const float *S, int64_t n, int k, const float *anchors, int n_anchor,
                               const uint32_t *grp, uint32_t *key, int num_sms, cudaStream_t st);
// Stable-within-key counting sort of rows by key < n_keys: perm[new] = old row.
cudaError_t launch_key_histogram(const uint32_t *key, int64_t n, uint32_t *hist, cudaStream_t st);
cudaError_t launch_key_scan(uint32_t *hist, int n_keys, cudaStream_t st);  // in place, exclusive
cudaError_t launch_key_scatter(const uint32_t *key, int64_t n, uint32_t *cursor, uint32_t *perm, cudaStream_t st);
// Row gathers: out row i <- in row perm[i] (bytes per row), and for vectors.
cudaError_t launch_gather_rows(const void *in, int64_t row_bytes, const uint32_t *perm, int64_t n, void *out,
                               cudaStream_t st);
cudaError_t launch_gather_u32(const uint32_t *in, const uint32_t *perm, int64_t n, uint32_t *out, cudaStream_t st);
cudaError_t launch_gather_f32(const float *in, const uint32_t *perm, int64_t n, float *out, cudaStream_t st);
// Covering anchors: drop[a] = 1 when an earlier candidate b < a has sketch cosine >= tau with
// candidate a (rows cand[] of S).
cudaError_t launch_cover_drop(const float *S, const uint32_t *cand, int nc, float tau, unsigned char *drop,
                              cudaStream_t st);
// covered[r] = 1 for each candidate (r, c) in cand[0 .. min(*count, cap)).
cudaError_t launch_cover_mark(const uint2 *cand, const unsigned long long *count, uint64_t cap,
                              unsigned char *covered, int num_sms, cudaStream_t st);
// Assignment of rows to covering anchors from the candidates (row, anchor) of a threshold
// contraction of the sketches against the anchors: best[r] = max over r's candidates of
// (cosine bits << 32 | anchor) (best zeroed by the caller); key[r] = its anchor, or n_anchor
// when no candidate reached row r.
cudaError_t launch_anchor_argmax(const uint2 *cand, const unsigned long long *cand_count, uint64_t cap, const float *S,
                                 const float *anchors, unsigned long long *best, int num_sms, cudaStream_t st);
cudaError_t launch_anchor_keys(const unsigned long long *best, int64_t n, int n_anchor, uint32_t *key, int num_sms,
                               cudaStream_t st);
// Tile-pair bounds on the tensor cores: rows of ball_k() FP32 columns whose dot product is >= 0 exactly when
// the ball pair's bound reaches eps_sketch (side 0: the A balls, with alpha = acos(eps_sketch) folded in;
// side 1: the B balls); rows n_balls .. rows_pad - 1 are zero padding.
int ball_k();
cudaError_t launch_ball_rows(const float *cent, const float *rad, int64_t n_balls, int64_t rows_pad,
                             float eps_sketch, int side, float *out, int num_sms, cudaStream_t st);
// The kept ball pairs (candidates of the threshold contraction of the two ball matrices) as the list of kept
// (A tile, B tile) pairs, ordered by A tile then B tile (bits: tA * tB bits, row_cnt: tA entries); sym: only
// block pairs on or above the diagonal.  *list_count = the number of kept tile pairs (the list holds the
// first list_cap).
cudaError_t launch_ball_pairs_to_list(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                      int64_t tA, int64_t tB, int sym, uint32_t *bits, uint32_t *row_cnt,
                                      uint2 *list, uint64_t list_cap, unsigned long long *list_count, int num_sms,
                                      cudaStream_t st);
// Balls per tile in the pruning bound.
constexpr int PRUNE_BALLS = 4;
// Per tile of `tile_rows` (<= 256) consecutive sketch rows: up to PRUNE_BALLS balls formed greedily
// along the row order: unit centroids [tiles x PRUNE_BALLS x 64] and angular radii
// [tiles x PRUNE_BALLS] (+ margin; -1 for an unused ball).
cudaError_t launch_tile_stats(const float *S, int64_t n, int k, int tile_rows, float *centroid, float *radius,
                              cudaStream_t st);
// Surviving tile pairs: some ball pair has cos(max(0, angle(c_a, c_b) - r_a - r_b)) >= eps_sketch.
// sym (self-join, A tiles of 128 and B tiles of 256 rows of one order): only pairs with a / 2 <= b.
cudaError_t launch_tile_pairs(const float *cA, const float *rA, int64_t tA, const float *cB, const float *rB,
                              int64_t tB, int k, float eps_sketch, uint2 *list, uint64_t cap,
                              unsigned long long *count, cudaStream_t st, int sym = 0);

}  // namespace ej
