// Top-k join condition (Sec. VI-E, the "top-k" vector join predicate; the paper evaluates k = 1
// and k = 32): for every kept R row, the k kept S rows of largest cosine similarity.
//
// The two contraction passes (sim_tc.cu, MODE_TOPMAX / MODE_TOPCAND) leave, per operand row r of
// A, every column whose bulk similarity lies within 2 * band of a lower bound of the row's k-th
// largest bulk similarity: since a bulk similarity is within band of the exact one, those columns
// hold the exact top k.  The kernels here finish the job:
//   * k > 1: the lower bound itself, the k-th largest of the row's column-group maxima (k groups
//     hold k distinct columns at or above it);
//   * the FP32 re-score of every candidate from the raw rows (the arithmetic of the threshold
//     re-score), packed with its column as one 64-bit key, f2ord(sim) << 32 | ~j, so that a larger
//     key is a larger similarity, then the smaller original j;
//   * k = 1: a 64-bit atomicMax of the key per row;  k > 1: a counting sort of the keys by row and
//     a per-row warp top-k (bitonic sort of each 32-key batch and merge into the running top 32).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ejoin_internal.cuh"

namespace ej {

namespace {

__device__ __forceinline__ unsigned long long pack_key(float sim, uint32_t j)
{
    return ((unsigned long long)f2ord(sim) << 32) | (unsigned long long)(~j);
}

__device__ __forceinline__ ejoin_pair unpack_key(unsigned long long key, uint32_t i)
{
    ejoin_pair p;
    p.i = i;
    p.j = ~(uint32_t)(key & 0xffffffffull);
    p.sim = ord2f((unsigned)(key >> 32));
    return p;
}

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int m)
{
    return __shfl_xor_sync(0xffffffffu, v, m);
}

// Bitonic sort of one key per lane into descending order across the warp (lane 0 the largest).
__device__ __forceinline__ unsigned long long warp_sort_desc(unsigned long long x, int lane)
{
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
        const bool desc = (lane & size) == 0;  // direction of this lane's block of `size` lanes
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const unsigned long long o = shfl_xor_u64(x, stride);
            const bool lower = (lane & stride) == 0;
            x = (lower == desc) ? (x > o ? x : o) : (x < o ? x : o);
        }
    }
    return x;
}

// Descending bitonic merge of a bitonic sequence held one key per lane.
__device__ __forceinline__ unsigned long long warp_merge_desc(unsigned long long x, int lane)
{
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        const unsigned long long o = shfl_xor_u64(x, stride);
        x = (lane & stride) == 0 ? (x > o ? x : o) : (x < o ? x : o);
    }
    return x;
}

// FP32 re-score of the candidates, one warp per 32 candidates: lane t fetches candidate t, then the
// warp gathers the rows of C candidates at once (V float4 per lane per row, every load issued before
// the first FMA: 2 * C * V independent loads in flight per lane) for rows of d <= 128 * V floats,
// 16-byte aligned; V = 0 is the general fallback (one candidate at a time, scalar loads).  Each
// lane ends with its candidate's key.  TOP1: atomicMax of the key into best[r]; otherwise the key
// is stored beside the candidate and row_cnt[r] counts it.
constexpr int RK_WARPS = 8;

template <int V, int C, bool TOP1>
__global__ void __launch_bounds__(RK_WARPS * 32) topk_rescore_kernel(
    const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_count, uint64_t cand_cap,
    const float *__restrict__ R, int64_t ldR, const float *__restrict__ S, int64_t ldS, int d,
    const uint32_t *__restrict__ idsR, const uint32_t *__restrict__ idsS, const float *__restrict__ invR,
    const float *__restrict__ invS, unsigned long long *__restrict__ out_keys, unsigned *__restrict__ row_cnt)
{
    const int lane = threadIdx.x & 31;
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    const int d4 = d >> 2;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = w0 * 32; base < n; base += nw * 32) {
        const bool valid = base + lane < n;
        uint32_t cr = 0, gi = 0, gj = 0;
        float sc = 0.f;
        if (valid) {
            const uint2 c = cand[base + lane];
            cr = c.x;
            gi = idsR ? idsR[c.x] : c.x;
            gj = idsS ? idsS[c.y] : c.y;
            sc = invR[c.x] * invS[c.y];
        }
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        float my_acc = 0.f;
        if constexpr (V > 0) {
#pragma unroll 1
            for (int q0 = 0; q0 < 32; q0 += C) {
                if (!((vmask >> q0) & 1u)) break;  // warp-uniform
                float4 a[C][V], b[C][V];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t ii = __shfl_sync(0xffffffffu, gi, q0 + c);
                    const uint32_t jj = __shfl_sync(0xffffffffu, gj, q0 + c);
                    const bool ok = (vmask >> (q0 + c)) & 1u;
                    const float4 *r = reinterpret_cast<const float4 *>(R + (int64_t)ii * ldR);
                    const float4 *s = reinterpret_cast<const float4 *>(S + (int64_t)jj * ldS);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int g = lane + 32 * v;
                        const bool in = ok && g < d4;
                        a[c][v] = in ? __ldg(r + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                        b[c][v] = in ? __ldg(s + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                float acc[C];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    acc[c] = 0.f;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        acc[c] = fmaf(a[c][v].x, b[c][v].x, acc[c]);
                        acc[c] = fmaf(a[c][v].y, b[c][v].y, acc[c]);
                        acc[c] = fmaf(a[c][v].z, b[c][v].z, acc[c]);
                        acc[c] = fmaf(a[c][v].w, b[c][v].w, acc[c]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
#pragma unroll
                for (int c = 0; c < C; ++c)
                    if (lane == q0 + c) my_acc = acc[c];
            }
        } else {
            for (int q = 0; q < 32; ++q) {
                if (!((vmask >> q) & 1u)) break;
                const uint32_t ii = __shfl_sync(0xffffffffu, gi, q);
                const uint32_t jj = __shfl_sync(0xffffffffu, gj, q);
                const float *r = R + (int64_t)ii * ldR, *s = S + (int64_t)jj * ldS;
                float acc = 0.f;
                for (int kk = lane; kk < d; kk += 32) acc = fmaf(__ldg(r + kk), __ldg(s + kk), acc);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == q) my_acc = acc;
            }
        }
        if (valid) {
            const unsigned long long key = pack_key(fminf(1.f, fmaxf(-1.f, my_acc * sc)), gj);
            if constexpr (TOP1) {
                atomicMax(out_keys + cr, key);
            } else {
                out_keys[base + lane] = key;
                atomicAdd(row_cnt + cr, 1u);
            }
        }
    }
}

// One record per kept R row, at its operand row r (so in ascending original i): every row has a
// best pair once S keeps a row, because pass 1 keeps the column that set the row's pass-0 maximum.
__global__ void top1_emit_kernel(const unsigned long long *__restrict__ best, const long long *__restrict__ nA_dev,
                                 int64_t nA_max, const uint32_t *__restrict__ idsR, ejoin_pair *__restrict__ out,
                                 uint64_t out_cap, unsigned long long *missing)
{
    int64_t n = *nA_dev;
    if (n > nA_max) n = nA_max;
    if ((uint64_t)n > out_cap) n = (int64_t)out_cap;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = best[r];
        const uint32_t i = idsR ? idsR[r] : (uint32_t)r;
        if (b) {
            out[r] = unpack_key(b, i);
        } else {
            out[r] = ejoin_pair{i, ~0u, -INFINITY};
            atomicAdd(missing, 1ull);
        }
    }
}

// Block per row: the k-th largest of the row's valid group maxima, found bit by bit from the top
// (the largest T with at least k values >= T is the k-th largest value).  Only the leading
// THR_BITS bits are searched: the result, with its low bits zero, is at most the k-th largest
// (a lower bound is all the candidate pass needs) and below it by less than 2^-11 relative.
constexpr int THR_BITS = 20;
constexpr int THR_THREADS = 256;

__global__ void __launch_bounds__(THR_THREADS) topk_threshold_kernel(const unsigned *__restrict__ gmax, int64_t ld,
                                                                     int shift, const long long *__restrict__ nA_dev,
                                                                     int64_t nA_max,
                                                                     const long long *__restrict__ nB_dev, int k,
                                                                     unsigned *__restrict__ thr)
{
    extern __shared__ unsigned sv[];  // ld values
    __shared__ unsigned wsum[2][THR_THREADS / 32];
    int64_t nA = *nA_dev;
    if (nA > nA_max) nA = nA_max;
    const long long nB = *nB_dev;
    int64_t G = nB <= 0 ? 0 : ((nB - 1) >> shift) + 1;
    if (G > ld) G = ld;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t r = blockIdx.x; r < nA; r += gridDim.x) {
        if (G < k) {  // fewer groups than k: every column is a candidate
            if (threadIdx.x == 0) thr[r] = f2ord(-INFINITY);
            continue;
        }
        for (int64_t g = threadIdx.x; g < G; g += THR_THREADS) sv[g] = gmax[r * ld + g];
        __syncthreads();
        unsigned res = 0u;
        for (int b = 31; b > 31 - THR_BITS; --b) {
            const unsigned cand = res | (1u << b);
            unsigned c = 0;
            for (int64_t g = threadIdx.x; g < G; g += THR_THREADS) c += sv[g] >= cand ? 1u : 0u;
            c = __reduce_add_sync(0xffffffffu, c);
            if (lane == 0) wsum[b & 1][warp] = c;
            __syncthreads();
            unsigned tot = 0;
#pragma unroll
            for (int w = 0; w < THR_THREADS / 32; ++w) tot += wsum[b & 1][w];
            if (tot >= (unsigned)k) res = cand;
        }
        // res == 0: fewer than k groups hold a value (a sampled first pass): no bound
        if (threadIdx.x == 0) thr[r] = res ? res : f2ord(-INFINITY);
        __syncthreads();  // sv is refilled for the next row
    }
}

__global__ void topk_scatter_kernel(const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_count,
                                    uint64_t cand_cap, const unsigned long long *__restrict__ keys,
                                    const unsigned *__restrict__ row_off, unsigned *__restrict__ row_fill,
                                    unsigned long long *__restrict__ seg)
{
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = cand[t].x;
        seg[(uint64_t)row_off[r] + atomicAdd(row_fill + r, 1u)] = keys[t];
    }
}

// Warp per row: lane t holds the row's (t+1)-th largest key so far.  A batch of 32 keys that holds
// none above the current kk-th is skipped; otherwise it is sorted and merged: max(best[t],
// batch[31 - t]) is a bitonic sequence holding the 32 largest of both, which one merge sorts.
__global__ void __launch_bounds__(256) topk_select_kernel(const unsigned long long *__restrict__ seg,
                                                          const unsigned *__restrict__ row_off,
                                                          const unsigned *__restrict__ row_cnt,
                                                          const long long *__restrict__ nA_dev, int64_t nA_max,
                                                          int kk, const uint32_t *__restrict__ idsR,
                                                          ejoin_pair *__restrict__ out, uint64_t out_cap,
                                                          unsigned long long *missing)
{
    const int lane = threadIdx.x & 31;
    int64_t nA = *nA_dev;
    if (nA > nA_max) nA = nA_max;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < nA; r += nw) {
        const unsigned n = row_cnt[r];
        const unsigned long long *src = seg + row_off[r];
        unsigned long long best = 0ull;  // 0 lies below every key
        for (unsigned b = 0; b < n; b += 32) {
            unsigned long long x = b + lane < n ? src[b + lane] : 0ull;
            const unsigned long long kth = shfl_u64(best, kk - 1);
            if (!__any_sync(0xffffffffu, x > kth)) continue;
            x = warp_sort_desc(x, lane);
            const unsigned long long rev = shfl_u64(x, 31 - lane);
            best = warp_merge_desc(best > rev ? best : rev, lane);
        }
        const uint32_t i = idsR ? idsR[r] : (uint32_t)r;
        const uint64_t slot = (uint64_t)r * kk + lane;
        if (lane < kk && slot < out_cap) {
            if (best) {
                out[slot] = unpack_key(best, i);
            } else {
                out[slot] = ejoin_pair{i, ~0u, -INFINITY};
                atomicAdd(missing, 1ull);
            }
        }
    }
}

unsigned grid_for(uint64_t work_items, uint64_t per_block, int num_sms, int blocks_per_sm)
{
    const uint64_t want = (work_items + per_block - 1) / per_block;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms * blocks_per_sm));
}

}  // namespace

namespace {

template <bool TOP1>
cudaError_t launch_rescore_keys(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                const float *R, int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *idsR,
                                const uint32_t *idsS, const float *invR, const float *invS, unsigned long long *keys,
                                unsigned *row_cnt, int num_sms, cudaStream_t st)
{
    if (cand_cap == 0) return cudaSuccess;
    const unsigned g = grid_for(cand_cap, RK_WARPS * 32, num_sms, 8);
    const int T = RK_WARPS * 32;
    const bool aligned = (d % 4 == 0) && (ldR % 4 == 0) && (ldS % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(R) % 16 == 0) && (reinterpret_cast<uintptr_t>(S) % 16 == 0);
#define EJ_RK_ARGS cand, cand_count, cand_cap, R, ldR, S, ldS, d, idsR, idsS, invR, invS, keys, row_cnt
    if (aligned && d <= 128) topk_rescore_kernel<1, 4, TOP1><<<g, T, 0, st>>>(EJ_RK_ARGS);
    else if (aligned && d <= 256) topk_rescore_kernel<2, 4, TOP1><<<g, T, 0, st>>>(EJ_RK_ARGS);
    else if (aligned && d <= 384) topk_rescore_kernel<3, 4, TOP1><<<g, T, 0, st>>>(EJ_RK_ARGS);
    else if (aligned && d <= 512) topk_rescore_kernel<4, 2, TOP1><<<g, T, 0, st>>>(EJ_RK_ARGS);
    else if (aligned && d <= 768) topk_rescore_kernel<6, 2, TOP1><<<g, T, 0, st>>>(EJ_RK_ARGS);
    else if (aligned && d <= 1024) topk_rescore_kernel<8, 2, TOP1><<<g, T, 0, st>>>(EJ_RK_ARGS);
    else topk_rescore_kernel<0, 1, TOP1><<<g, T, 0, st>>>(EJ_RK_ARGS);
#undef EJ_RK_ARGS
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_top1_rescore(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                const float *R, int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *idsR,
                                const uint32_t *idsS, const float *invR, const float *invS, unsigned long long *best,
                                int num_sms, cudaStream_t st)
{
    return launch_rescore_keys<true>(cand, cand_count, cand_cap, R, ldR, S, ldS, d, idsR, idsS, invR, invS, best,
                                     nullptr, num_sms, st);
}

cudaError_t launch_top1_emit(const unsigned long long *best, const long long *nA_dev, int64_t nA_max,
                             const uint32_t *idsR, ejoin_pair *out, uint64_t out_cap, unsigned long long *missing,
                             int num_sms, cudaStream_t st)
{
    if (nA_max <= 0 || out_cap == 0) return cudaSuccess;
    top1_emit_kernel<<<grid_for(nA_max, 256, num_sms, 8), 256, 0, st>>>(best, nA_dev, nA_max, idsR, out, out_cap,
                                                                      missing);
    return cudaGetLastError();
}

cudaError_t launch_topk_threshold(const unsigned *gmax, int64_t ld, int shift, const long long *nA_dev,
                                  int64_t nA_max, const long long *nB_dev, int k, unsigned *thr, int num_sms,
                                  cudaStream_t st)
{
    if (nA_max <= 0) return cudaSuccess;
    if (ld <= 0 || ld > TOPK_MAX_GROUPS || k < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)ld * sizeof(unsigned);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(topk_threshold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    topk_threshold_kernel<<<grid_for(nA_max, 1, num_sms, 8), THR_THREADS, smem, st>>>(gmax, ld, shift, nA_dev,
                                                                                     nA_max, nB_dev, k, thr);
    return cudaGetLastError();
}

cudaError_t launch_topk_rescore(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                const float *R, int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *idsR,
                                const uint32_t *idsS, const float *invR, const float *invS, unsigned long long *keys,
                                unsigned *row_cnt, int num_sms, cudaStream_t st)
{
    return launch_rescore_keys<false>(cand, cand_count, cand_cap, R, ldR, S, ldS, d, idsR, idsS, invR, invS, keys,
                                      row_cnt, num_sms, st);
}

cudaError_t launch_topk_scatter(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                const unsigned long long *keys, const unsigned *row_off, unsigned *row_fill,
                                unsigned long long *seg, int num_sms, cudaStream_t st)
{
    if (cand_cap == 0) return cudaSuccess;
    topk_scatter_kernel<<<grid_for(cand_cap, 256, num_sms, 8), 256, 0, st>>>(cand, cand_count, cand_cap, keys, row_off,
                                                                           row_fill, seg);
    return cudaGetLastError();
}

cudaError_t launch_topk_select(const unsigned long long *seg, const unsigned *row_off, const unsigned *row_cnt,
                               const long long *nA_dev, int64_t nA_max, int kk, const uint32_t *idsR, ejoin_pair *out,
                               uint64_t out_cap, unsigned long long *missing, int num_sms, cudaStream_t st)
{
    if (nA_max <= 0 || out_cap == 0) return cudaSuccess;
    if (kk < 1 || kk > 32) return cudaErrorInvalidValue;
    topk_select_kernel<<<grid_for(nA_max, 8, num_sms, 8), 256, 0, st>>>(seg, row_off, row_cnt, nA_dev, nA_max, kk,
                                                                      idsR, out, out_cap, missing);
    return cudaGetLastError();
}

}  // namespace ej
