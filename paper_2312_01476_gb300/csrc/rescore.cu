// Exact re-score of the contraction's candidates (guard band around eps).
//
// Every candidate (a pair whose bulk-precision similarity reached eps - band)
// gets its similarity recomputed from the original FP32 rows (Sec. III-A,
// Eq. (Cosine Similarity)): an FP32 dot product, lane-parallel with a
// butterfly reduction, scaled by the two FP32 inverse norms from the
// normalisation pass.  A candidate whose FP32 similarity lies within
// fp64_band of eps is recomputed by the accurate tier (compensated dot
// product and both norms, finished in FP64; accurate_cosine).
// Pairs with sim >= eps (Sec. III-B threshold predicate) are emitted as
// (original i, original j, sim) records (Sec. IV-C, mapping back to tuples),
// one global atomic per block of candidates.
#include <algorithm>

#include "ejoin_internal.cuh"

namespace ej {

namespace {
constexpr int RS_WARPS = 8;
constexpr int RS_PER_WARP = 16;  // candidates per warp per block step
constexpr int RS_PER_BLOCK = RS_WARPS * RS_PER_WARP;
}  // namespace

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


// Block-level aggregation of the re-score's outcomes (lane q of each warp holds
// one candidate's result): one global atomic per block step.  mirror (a
// self-join evaluated on the upper triangle only): a pair (i, j) with i != j
// is written as (i, j) and (j, i), both with the same similarity, which is
// exact because the FP32 dot product and the accurate tier are symmetric in
// their two rows.
template <bool MIRROR>
__device__ __forceinline__ void emit_block(bool my_emit, uint32_t my_i, uint32_t my_j, float my_sim, int *wcnt,
                                           unsigned long long *base_s, unsigned long long *out_count,
                                           ejoin_pair *__restrict__ out, uint64_t out_cap, int count_only, int lane,
                                           int warp)
{
    int mine, incl;
    if constexpr (MIRROR) {
        mine = my_emit ? (my_i != my_j ? 2 : 1) : 0;
        incl = mine;  // warp inclusive scan of the record counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, my_emit);
    if (lane == 0) {
        if constexpr (MIRROR) {
            wcnt[warp] = 0;
        } else {
            wcnt[warp] = __popc(m);
        }
    }
    if constexpr (MIRROR) {
        if (lane == 31) wcnt[warp] = incl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < RS_WARPS; ++w) {
            const int c = wcnt[w];
            wcnt[w] = run;
            run += c;
        }
        *base_s = run ? atomicAdd(out_count, (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    if (my_emit && !count_only) {
        unsigned long long pos;
        if constexpr (MIRROR) pos = *base_s + (unsigned long long)(wcnt[warp] + incl - mine);
        else pos = *base_s + wcnt[warp] + __popc(m & ((1u << lane) - 1u));
        if (pos < out_cap) {
            ejoin_pair p;
            p.i = my_i;
            p.j = my_j;
            p.sim = my_sim;
            out[pos] = p;
        }
        if constexpr (MIRROR) {
            if (mine == 2 && pos + 1 < out_cap) {
                ejoin_pair p;
                p.i = my_j;
                p.j = my_i;
                p.sim = my_sim;
                out[pos + 1] = p;
            }
        }
    }
    __syncthreads();
}

template <bool MIRROR>
__global__ void __launch_bounds__(RS_WARPS * 32) rescore_kernel(
    const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_count, uint64_t cand_cap,
    const float *__restrict__ R, int64_t ldR, const float *__restrict__ S, int64_t ldS, int d,
    const uint32_t *__restrict__ idsR, const uint32_t *__restrict__ idsS, const float *__restrict__ invR,
    const float *__restrict__ invS, float eps, float fp64_band, ejoin_pair *__restrict__ out, uint64_t out_cap,
    unsigned long long *out_count, unsigned long long *band_count, int count_only, uint2 *__restrict__ band_list,
    uint64_t band_cap)
{
    __shared__ int wcnt[RS_WARPS];
    __shared__ unsigned long long base_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    const bool vec = ((ldR & 3) == 0) && ((ldS & 3) == 0) && ((reinterpret_cast<uintptr_t>(R) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(S) & 15) == 0);
    const int d4 = vec ? (d >> 2) : 0;  // float4 groups
    for (uint64_t start = (uint64_t)blockIdx.x * RS_PER_BLOCK; start < n;
         start += (uint64_t)gridDim.x * RS_PER_BLOCK) {
        const int len = (int)std::min<uint64_t>(RS_PER_BLOCK, n - start);
        // lane q (< RS_PER_WARP) holds the outcome of the warp's q-th candidate
        bool my_emit = false;
        uint32_t my_i = 0, my_j = 0;
        float my_sim = 0.f;
        const int wofs = warp * RS_PER_WARP;
        const uint64_t wbase = start + (uint64_t)wofs;
        for (int q = 0; q < RS_PER_WARP; ++q) {
            const uint64_t k = wbase + q;
            if (wofs + q >= len) break;  // warp-uniform
            const uint2 c = cand[k];
            const uint32_t i = idsR ? idsR[c.x] : c.x;
            const uint32_t j = idsS ? idsS[c.y] : c.y;
            const float *r = R + (int64_t)i * ldR;
            const float *s = S + (int64_t)j * ldS;
            float acc = 0.f;
            for (int g = lane; g < d4; g += 32) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(r) + g);
                const float4 b = __ldg(reinterpret_cast<const float4 *>(s) + g);
                acc = fmaf(a.x, b.x, acc);
                acc = fmaf(a.y, b.y, acc);
                acc = fmaf(a.z, b.z, acc);
                acc = fmaf(a.w, b.w, acc);
            }
            for (int kk = 4 * d4 + lane; kk < d; kk += 32) acc = fmaf(__ldg(r + kk), __ldg(s + kk), acc);
            acc = warp_sum_f(acc);
            float sim = acc * invR[c.x] * invS[c.y];
            sim = fminf(1.f, fmaxf(-1.f, sim));
            bool emit = sim >= eps;
            if (fabsf(sim - eps) < fp64_band) {
                // near eps: decided by the accurate tier (rescore_band_kernel)
                if (lane == 0) {
                    const unsigned long long p = atomicAdd(band_count, 1ull);
                    if (p < band_cap) band_list[p] = make_uint2(i, j);
                }
                emit = false;
            }
            if (lane == q) {
                my_emit = emit;
                my_i = i;
                my_j = j;
                my_sim = sim;
            }
        }
        emit_block<MIRROR>(my_emit, my_i, my_j, my_sim, wcnt, &base_s, out_count, out, out_cap, count_only, lane,
                           warp);
    }
}

// Variant for d <= 128 * V with 16-byte aligned rows: each warp gathers the
// rows of C candidates at once (V float4 per lane per row, all loads issued
// before the first FMA), so that 2*C*V independent loads are in flight per
// lane instead of a dependent chain per candidate.
template <int V, int C, bool MIRROR, bool FENCE>
__global__ void __launch_bounds__(RS_WARPS * 32) rescore_mlp_kernel(
    const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_count, uint64_t cand_cap,
    const float *__restrict__ R, int64_t ldR, const float *__restrict__ S, int64_t ldS, int d,
    const uint32_t *__restrict__ idsR, const uint32_t *__restrict__ idsS, const float *__restrict__ invR,
    const float *__restrict__ invS, float eps, float fp64_band, ejoin_pair *__restrict__ out, uint64_t out_cap,
    unsigned long long *out_count, unsigned long long *band_count, int count_only, uint2 *__restrict__ band_list,
    uint64_t band_cap)
{
    static_assert(RS_PER_WARP % C == 0, "candidates per warp step");
    __shared__ int wcnt[RS_WARPS];
    __shared__ unsigned long long base_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    const int d4 = d >> 2;  // d is a multiple of 4 here
    for (uint64_t start = (uint64_t)blockIdx.x * RS_PER_BLOCK; start < n;
         start += (uint64_t)gridDim.x * RS_PER_BLOCK) {
        const int len = (int)std::min<uint64_t>(RS_PER_BLOCK, n - start);
        bool my_emit = false;
        uint32_t my_i = 0, my_j = 0;
        float my_sim = 0.f;
        const int wofs = warp * RS_PER_WARP;
        const uint64_t wbase = start + (uint64_t)wofs;
        // lanes 0..RS_PER_WARP-1 fetch the warp's candidates and their ids / inverse norms
        uint32_t ci = 0, cj = 0, gi = 0, gj = 0;
        float sc = 0.f;
        bool valid = false;
        if (lane < RS_PER_WARP && wofs + lane < len) {
            const uint2 c = cand[wbase + lane];
            ci = c.x;
            cj = c.y;
            gi = idsR ? idsR[ci] : ci;
            gj = idsS ? idsS[cj] : cj;
            sc = invR[ci] * invS[cj];
            valid = true;
        }
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        // symmetric self-joins (dense tiles): the R row of the previous candidate, kept in registers, since
        // consecutive candidates often share it (a lane of the contraction epilogue emits its row's matches
        // of a chunk together).  Sparse candidate lists gain nothing and would pay the registers.
        constexpr bool REUSE = MIRROR;
        uint32_t prev_i = 0xffffffffu;
        float4 a_prev[V];
#pragma unroll
        for (int v = 0; v < V; ++v) a_prev[v] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
        for (int q0 = 0; q0 < RS_PER_WARP; q0 += C) {
            if (!((vmask >> q0) & 1u)) break;  // warp-uniform
            float4 a[C][V], b[C][V];
            uint32_t ii[C], jj[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                ii[c] = __shfl_sync(0xffffffffu, gi, q0 + c);
                jj[c] = __shfl_sync(0xffffffffu, gj, q0 + c);
                const bool ok = (vmask >> (q0 + c)) & 1u;
                const bool same = REUSE && ok && ii[c] == (c == 0 ? prev_i : ii[c - 1]);  // warp-uniform
                const float4 *r = reinterpret_cast<const float4 *>(R + (int64_t)ii[c] * ldR);
                const float4 *s = reinterpret_cast<const float4 *>(S + (int64_t)jj[c] * ldS);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int g = lane + 32 * v;
                    const bool in = ok && g < d4;
                    if (same)
                        a[c][v] = c == 0 ? a_prev[v] : a[c > 0 ? c - 1 : 0][v];
                    else
                        a[c][v] = in ? __ldg(r + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                    b[c][v] = in ? __ldg(s + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            // FENCE: without it the compiler consumes each candidate's rows before loading the next
            // candidate's (38 registers at V = 3, C = 4), so a warp waits for one gather after another.
            // A CTA-scope fence after the loads keeps all 2 C V of them in flight together (C = 2 at
            // V = 3: 63 registers); on the 1M x 100k d = 300 join this cut the re-score from 1.98 to 1.41 ms.
            if constexpr (FENCE) asm volatile("membar.cta;" ::: "memory");
            if constexpr (REUSE) {
                prev_i = ((vmask >> (q0 + C - 1)) & 1u) ? ii[C - 1] : 0xffffffffu;
#pragma unroll
                for (int v = 0; v < V; ++v) a_prev[v] = a[C - 1][v];
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
            for (int c = 0; c < C; ++c) {
                const int q = q0 + c;
                if (!((vmask >> q) & 1u)) break;
                float sim = acc[c] * __shfl_sync(0xffffffffu, sc, q);
                sim = fminf(1.f, fmaxf(-1.f, sim));
                bool emit = sim >= eps;
                if (fabsf(sim - eps) < fp64_band) {
                    // near eps: decided by the accurate tier (rescore_band_kernel)
                    if (lane == 0) {
                        const unsigned long long p = atomicAdd(band_count, 1ull);
                        if (p < band_cap) band_list[p] = make_uint2(ii[c], jj[c]);
                    }
                    emit = false;
                }
                if (lane == q) {
                    my_emit = emit;
                    my_i = ii[c];
                    my_j = jj[c];
                    my_sim = sim;
                }
            }
        }
        emit_block<MIRROR>(my_emit, my_i, my_j, my_sim, wcnt, &base_s, out_count, out, out_cap, count_only, lane,
                           warp);
    }
}

// Accurate tier of the re-score: the candidates that the FP32 tier found within
// fp64_band of eps, listed as (original i, original j), decided by
// accurate_cosine (compensated dot products finished in FP64).  One warp per
// entry, 32 entries per warp step, one global atomic per step.
template <bool MIRROR, bool VEC>
__global__ void __launch_bounds__(256) rescore_band_kernel(const uint2 *__restrict__ band_list,
                                                           const unsigned long long *__restrict__ band_count,
                                                           uint64_t band_cap, const float *__restrict__ R, int64_t ldR,
                                                           const float *__restrict__ S, int64_t ldS, int d, float eps,
                                                           ejoin_pair *__restrict__ out, uint64_t out_cap,
                                                           unsigned long long *out_count, int count_only)
{
    const int lane = threadIdx.x & 31;
    uint64_t n = *band_count;
    if (n > band_cap) n = band_cap;
    const double eps_d = (double)eps;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = w0 * 32; base < n; base += nw * 32) {
        const int len = (int)(n - base < 32 ? n - base : 32);
        const uint2 mine_e = lane < len ? band_list[base + lane] : make_uint2(0u, 0u);
        bool my_emit = false;
        float my_sim = 0.f;
        for (int q = 0; q < len; ++q) {
            const uint32_t i = __shfl_sync(0xffffffffu, mine_e.x, q), j = __shfl_sync(0xffffffffu, mine_e.y, q);
            const double s64 = VEC ? accurate_cosine4(R + (int64_t)i * ldR, S + (int64_t)j * ldS, d, lane)
                                   : accurate_cosine(R + (int64_t)i * ldR, S + (int64_t)j * ldS, d, lane);
            if (lane == q) {
                my_emit = s64 >= eps_d;
                my_sim = (float)s64;
            }
        }
        const int mine = my_emit ? ((MIRROR && mine_e.x != mine_e.y) ? 2 : 1) : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long pos0 = 0;
        if (lane == 0 && tot) pos0 = atomicAdd(out_count, (unsigned long long)tot);
        pos0 = __shfl_sync(0xffffffffu, pos0, 0);
        if (mine && !count_only) {
            const unsigned long long pos = pos0 + (unsigned long long)(incl - mine);
            ejoin_pair p;
            p.i = mine_e.x;
            p.j = mine_e.y;
            p.sim = my_sim;
            if (pos < out_cap) out[pos] = p;
            if (mine == 2 && pos + 1 < out_cap) {
                p.i = mine_e.y;
                p.j = mine_e.x;
                out[pos + 1] = p;
            }
        }
    }
}

// Accurate tier with per-row norms (BandNorms): the squared norms of the listed candidates' rows once, then
// each entry's cross product only.
// The squared norms of the rows the band list names, one warp per entry and side: the first warp to reach
// a row claims it (flag 0 -> 1, the flags cleared before the list is written) and computes its norm, so the
// work follows the list, not the relations' sizes.
template <bool VEC>
__global__ void __launch_bounds__(256) band_norm_kernel(const uint2 *__restrict__ band_list,
                                                        const unsigned long long *__restrict__ band_count,
                                                        uint64_t band_cap, const float *__restrict__ R, int64_t ldR,
                                                        const float *__restrict__ S, int64_t ldS, int d,
                                                        unsigned *claimR, unsigned *claimS, double *nrmR, double *nrmS)
{
    const int lane = threadIdx.x & 31;
    uint64_t n = *band_count;
    if (n > band_cap) n = band_cap;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t k = w0; k < 2 * n; k += nw) {
        const bool side_s = k >= n;
        const uint2 e = band_list[side_s ? k - n : k];
        const uint32_t row = side_s ? e.y : e.x;
        unsigned won = 0;
        if (lane == 0) won = atomicExch(side_s ? claimS + row : claimR + row, 1u) == 0u;
        won = __shfl_sync(0xffffffffu, won, 0);
        if (!won) continue;  // warp-uniform
        const float *x = side_s ? S + (int64_t)row * ldS : R + (int64_t)row * ldR;
        const double v = accurate_dot<VEC>(x, x, d, lane);
        if (lane == 0) (side_s ? nrmS : nrmR)[row] = v;
    }
}

template <bool MIRROR, bool VEC>
__global__ void __launch_bounds__(256) rescore_band_norms_kernel(
    const uint2 *__restrict__ band_list, const unsigned long long *__restrict__ band_count, uint64_t band_cap,
    const float *__restrict__ R, int64_t ldR, const float *__restrict__ S, int64_t ldS, int d,
    const double *__restrict__ nrmR, const double *__restrict__ nrmS, float eps, ejoin_pair *__restrict__ out,
    uint64_t out_cap, unsigned long long *out_count, int count_only)
{
    const int lane = threadIdx.x & 31;
    uint64_t n = *band_count;
    if (n > band_cap) n = band_cap;
    const double eps_d = (double)eps;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = w0 * 32; base < n; base += nw * 32) {
        const int len = (int)(n - base < 32 ? n - base : 32);
        const uint2 mine_e = lane < len ? band_list[base + lane] : make_uint2(0u, 0u);
        const double my_nr = lane < len ? nrmR[mine_e.x] : 0.0, my_ns = lane < len ? nrmS[mine_e.y] : 0.0;
        bool my_emit = false;
        float my_sim = 0.f;
        for (int q = 0; q < len; ++q) {
            const uint32_t i = __shfl_sync(0xffffffffu, mine_e.x, q), j = __shfl_sync(0xffffffffu, mine_e.y, q);
            const double dd = accurate_dot<VEC>(R + (int64_t)i * ldR, S + (int64_t)j * ldS, d, lane);
            if (lane == q) {
                // the expression of accurate_cosine, with the norms computed once per row
                double c = (my_nr > 0.0 && my_ns > 0.0) ? dd / (sqrt(my_nr) * sqrt(my_ns)) : 0.0;
                c = fmin(1.0, fmax(-1.0, c));
                my_emit = c >= eps_d;
                my_sim = (float)c;
            }
        }
        const int mine = my_emit ? ((MIRROR && mine_e.x != mine_e.y) ? 2 : 1) : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long pos0 = 0;
        if (lane == 0 && tot) pos0 = atomicAdd(out_count, (unsigned long long)tot);
        pos0 = __shfl_sync(0xffffffffu, pos0, 0);
        if (mine && !count_only) {
            const unsigned long long pos = pos0 + (unsigned long long)(incl - mine);
            ejoin_pair p;
            p.i = mine_e.x;
            p.j = mine_e.y;
            p.sim = my_sim;
            if (pos < out_cap) out[pos] = p;
            if (mine == 2 && pos + 1 < out_cap) {
                p.i = mine_e.y;
                p.j = mine_e.x;
                out[pos + 1] = p;
            }
        }
    }
}

// Batched re-score: candidate (a, b) holds rows of the concatenated operands;
// job j owns a in [a_off[j], a_off[j+1]) and b in [b_off[j], b_off[j+1]).  The
// FP32 rows are read from the job's own input (row a - a_off[j] of R_j, row
// b - b_off[j] of S_j) and the job's eps decides; records are (job, i, j, sim).
// V > 0: rows gathered as V float4 per lane (16-byte aligned inputs, d % 4 == 0,
// d <= 128 V); V == 0: scalar loop for any d and alignment.
template <int V>
__global__ void __launch_bounds__(RS_WARPS * 32, 2) rescore_batch_kernel(
    const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_count, uint64_t cand_cap,
    const BatchRows br, int d, const float *__restrict__ invA, const float *__restrict__ invB, float fp64_band,
    BatchPair *__restrict__ out, uint64_t out_cap, unsigned long long *out_count, unsigned long long *band_count)
{
    __shared__ int wcnt[RS_WARPS];
    __shared__ unsigned long long base_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    const int d4 = d >> 2;

    for (uint64_t blk = (uint64_t)blockIdx.x * RS_PER_BLOCK; blk < n; blk += (uint64_t)gridDim.x * RS_PER_BLOCK) {
        bool my_emit = false;
        BatchPair my{};
        int my_band = 0;
        const uint64_t wbase = blk + (uint64_t)warp * RS_PER_WARP;
        // lanes 0..RS_PER_WARP-1 resolve the warp's candidates: job, local ids, scale, eps
        uint32_t gi = 0, gj = 0, job = 0;
        float sc = 0.f, ej = 0.f;
        bool valid = false;
        if (lane < RS_PER_WARP && wbase + lane < n) {
            const uint2 c = cand[wbase + lane];
            int lo = 0, hi = br.n_jobs;  // a_off[lo] <= c.x < a_off[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(br.a_off + mid) <= (long long)c.x) lo = mid;
                else hi = mid;
            }
            job = (uint32_t)lo;
            gi = batch_row_a(br, c.x, job);
            gj = batch_row_b(br, c.y, job);
            sc = invA[c.x] * invB[c.y];
            ej = __ldg(br.eps + lo);
            valid = true;
        }
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        // C candidates per step: their rows are gathered together (2 C V loads in flight per lane), then
        // summed and decided one by one
        constexpr int C = V == 0 ? 1 : (V <= 3 ? 4 : 2);
        static_assert(RS_PER_WARP % C == 0, "candidates per warp step");
#pragma unroll 1
        for (int q0 = 0; q0 < RS_PER_WARP; q0 += C) {
            if (!((vmask >> q0) & 1u)) break;  // warp-uniform
            uint32_t jb[C], ii[C], jj[C];
            const float *rp[C], *sp[C];
            float acc[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const bool ok = (vmask >> (q0 + c)) & 1u;
                jb[c] = __shfl_sync(0xffffffffu, job, q0 + c);
                ii[c] = __shfl_sync(0xffffffffu, gi, q0 + c);
                jj[c] = __shfl_sync(0xffffffffu, gj, q0 + c);
                rp[c] = ok ? br.R[jb[c]] + (int64_t)ii[c] * br.ldR[jb[c]] : nullptr;
                sp[c] = ok ? br.S[jb[c]] + (int64_t)jj[c] * br.ldS[jb[c]] : nullptr;
                acc[c] = 0.f;
            }
            if constexpr (V > 0) {
                float4 a[C][V], b[C][V];
#pragma unroll
                for (int c = 0; c < C; ++c) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int g = lane + 32 * v;
                        const bool in = rp[c] != nullptr && g < d4;
                        a[c][v] = in ? __ldg(reinterpret_cast<const float4 *>(rp[c]) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                        b[c][v] = in ? __ldg(reinterpret_cast<const float4 *>(sp[c]) + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        acc[c] = fmaf(a[c][v].x, b[c][v].x, acc[c]);
                        acc[c] = fmaf(a[c][v].y, b[c][v].y, acc[c]);
                        acc[c] = fmaf(a[c][v].z, b[c][v].z, acc[c]);
                        acc[c] = fmaf(a[c][v].w, b[c][v].w, acc[c]);
                    }
            } else {
                if (rp[0])
                    for (int kk = lane; kk < d; kk += 32) acc[0] = fmaf(__ldg(rp[0] + kk), __ldg(sp[0] + kk), acc[0]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int q = q0 + c;
                if (!((vmask >> q) & 1u)) break;  // warp-uniform
                const float eps = __shfl_sync(0xffffffffu, ej, q);
                float sim = fminf(1.f, fmaxf(-1.f, acc[c] * __shfl_sync(0xffffffffu, sc, q)));
                bool emit = sim >= eps;
                int band = 0;
                if (fabsf(sim - eps) < fp64_band) {
                    // accurate tier: compensated dot product and norms, finished in FP64
                    const double s64 = accurate_cosine(rp[c], sp[c], d, lane);
                    emit = s64 >= (double)eps;
                    sim = (float)s64;
                    band = 1;
                }
                if (lane == q) {
                    my_emit = emit;
                    my.job = jb[c];
                    my.i = ii[c];
                    my.j = jj[c];
                    my.sim = sim;
                    my_band = band;
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, my_emit);
        const int nb = __popc(__ballot_sync(0xffffffffu, my_band != 0));
        if (lane == 0) {
            wcnt[warp] = __popc(m);
            if (nb) atomicAdd(band_count, (unsigned long long)nb);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int w = 0; w < RS_WARPS; ++w) {
                const int c = wcnt[w];
                wcnt[w] = run;
                run += c;
            }
            base_s = run ? atomicAdd(out_count, (unsigned long long)run) : 0ull;
        }
        __syncthreads();
        if (my_emit) {
            const unsigned long long pos = base_s + wcnt[warp] + __popc(m & ((1u << lane) - 1u));
            if (pos < out_cap) out[pos] = my;
        }
        __syncthreads();
    }
}

cudaError_t launch_rescore_batch(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                 const BatchRows &br, int d, const float *invA, const float *invB, float fp64_band,
                                 BatchPair *out, uint64_t out_cap, unsigned long long *out_count,
                                 unsigned long long *band_count, bool aligned, int num_sms, cudaStream_t st)
{
    if (cand_cap == 0) return cudaSuccess;
    uint64_t blocks = (cand_cap + RS_PER_BLOCK - 1) / RS_PER_BLOCK;
    const uint64_t lim = (uint64_t)num_sms * 8;
    if (blocks > lim) blocks = lim;
    const unsigned g = (unsigned)blocks;
    const int T = RS_WARPS * 32;
    // `aligned`: every job's rows start on 16 bytes and d % 4 == 0 (checked by the host)
#define EJ_RB_ARGS cand, cand_count, cand_cap, br, d, invA, invB, fp64_band, out, out_cap, out_count, band_count
    if (aligned && d <= 128) rescore_batch_kernel<1><<<g, T, 0, st>>>(EJ_RB_ARGS);
    else if (aligned && d <= 256) rescore_batch_kernel<2><<<g, T, 0, st>>>(EJ_RB_ARGS);
    else if (aligned && d <= 384) rescore_batch_kernel<3><<<g, T, 0, st>>>(EJ_RB_ARGS);
    else if (aligned && d <= 512) rescore_batch_kernel<4><<<g, T, 0, st>>>(EJ_RB_ARGS);
    else if (aligned && d <= 768) rescore_batch_kernel<6><<<g, T, 0, st>>>(EJ_RB_ARGS);
    else if (aligned && d <= 1024) rescore_batch_kernel<8><<<g, T, 0, st>>>(EJ_RB_ARGS);
    else rescore_batch_kernel<0><<<g, T, 0, st>>>(EJ_RB_ARGS);
#undef EJ_RB_ARGS
    return cudaGetLastError();
}

// Exact FP32 cosine similarity of given pairs (one warp per pair): the
// re-score's FP32 tier without the threshold, used to label training pairs.
__global__ void score_pairs_kernel(const float *__restrict__ R, int64_t ldR, const float *__restrict__ S, int64_t ldS,
                                   int d, const uint32_t *__restrict__ pi, const uint32_t *__restrict__ pj,
                                   const float *__restrict__ invR, const float *__restrict__ invS, int64_t n,
                                   float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w; k < n; k += nw) {
        const uint32_t i = pi[k], j = pj[k];
        const float *r = R + (int64_t)i * ldR, *s = S + (int64_t)j * ldS;
        float acc = 0.f;
        for (int c = lane; c < d; c += 32) acc = fmaf(__ldg(r + c), __ldg(s + c), acc);
        acc = warp_sum_f(acc);
        if (lane == 0) out[k] = fminf(1.f, fmaxf(-1.f, acc * invR[i] * invS[j]));
    }
}

cudaError_t launch_score_pairs(const float *R, int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *pi,
                               const uint32_t *pj, const float *invR, const float *invS, int64_t n, float *out,
                               int num_sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 7) / 8;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    score_pairs_kernel<<<(unsigned)blocks, 256, 0, st>>>(R, ldR, S, ldS, d, pi, pj, invR, invS, n, out);
    return cudaGetLastError();
}

// The accurate tier over the candidates that the FP32 tier listed near eps (stream order: after it).
static cudaError_t launch_band_tier(const uint2 *band_list, const unsigned long long *band_count, uint64_t band_cap,
                                    const float *R, int64_t ldR, const float *S, int64_t ldS, int d, float eps,
                                    ejoin_pair *out, uint64_t out_cap, unsigned long long *out_count, int count_only,
                                    bool aligned, bool mirror, int num_sms, cudaStream_t st,
                                    const BandNorms *bn = nullptr)
{
    const unsigned gb = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((band_cap + 255) / 256, (uint64_t)num_sms * 8));
    if (bn) {
        cudaError_t e = cudaMemsetAsync(bn->claimR, 0, (size_t)(bn->nR + bn->nS) * 4, st);
        if (e != cudaSuccess) return e;
        const unsigned gn = (unsigned)std::max<uint64_t>(
            1, std::min<uint64_t>((2 * band_cap + 7) / 8, (uint64_t)num_sms * 16));
        if (aligned)
            band_norm_kernel<true><<<gn, 256, 0, st>>>(band_list, band_count, band_cap, R, ldR, S, ldS, d, bn->claimR,
                                                       bn->claimS, bn->nrmR, bn->nrmS);
        else
            band_norm_kernel<false><<<gn, 256, 0, st>>>(band_list, band_count, band_cap, R, ldR, S, ldS, d,
                                                        bn->claimR, bn->claimS, bn->nrmR, bn->nrmS);
#define EJ_BANDN(M, V)                                                                                            \
    rescore_band_norms_kernel<M, V><<<gb, 256, 0, st>>>(band_list, band_count, band_cap, R, ldR, S, ldS, d,        \
                                                       bn->nrmR, bn->nrmS, eps, out, out_cap, out_count, count_only)
        if (mirror) {
            if (aligned) EJ_BANDN(true, true);
            else EJ_BANDN(true, false);
        } else {
            if (aligned) EJ_BANDN(false, true);
            else EJ_BANDN(false, false);
        }
#undef EJ_BANDN
        return cudaGetLastError();
    }
#define EJ_BAND(M, V)                                                                                               \
    rescore_band_kernel<M, V><<<gb, 256, 0, st>>>(band_list, band_count, band_cap, R, ldR, S, ldS, d, eps, out, out_cap, \
                                                  out_count, count_only)
    if (mirror) {
        if (aligned) EJ_BAND(true, true);
        else EJ_BAND(true, false);
    } else {
        if (aligned) EJ_BAND(false, true);
        else EJ_BAND(false, false);
    }
#undef EJ_BAND
    return cudaGetLastError();
}

cudaError_t launch_rescore(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap, const float *R,
                           int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *idsR,
                           const uint32_t *idsS, const float *invR, const float *invS, float eps, float fp64_band,
                           ejoin_pair *out, uint64_t out_cap, unsigned long long *out_count,
                           unsigned long long *band_count, int count_only, int num_sms, cudaStream_t st,
                           uint2 *band_list, uint64_t band_cap, int mirror, const BandNorms *bn)
{
    if (cand_cap == 0) return cudaSuccess;
    // every candidate may fall in the band: the list must hold them all
    if (fp64_band > 0.f && (!band_list || band_cap < cand_cap)) return cudaErrorInvalidValue;
    uint64_t blocks = (cand_cap + RS_PER_BLOCK - 1) / RS_PER_BLOCK;
    const uint64_t lim = (uint64_t)num_sms * 8;
    if (blocks > lim) blocks = lim;
    const bool aligned = (d % 4 == 0) && (ldR % 4 == 0) && (ldS % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(R) % 16 == 0) && (reinterpret_cast<uintptr_t>(S) % 16 == 0);
    const unsigned g = (unsigned)blocks;
    const int T = RS_WARPS * 32;
#define EJ_RESCORE_ARGS                                                                                              \
    cand, cand_count, cand_cap, R, ldR, S, ldS, d, idsR, idsS, invR, invS, eps, fp64_band, out, out_cap, out_count, \
        band_count, count_only, band_list, band_cap
    // fenced gathers, C chosen so that at most 12 float4 of row data per lane are in flight
#define EJ_DISPATCH(M)                                                                                              \
    if (aligned && d <= 128) rescore_mlp_kernel<1, 4, M, true><<<g, T, 0, st>>>(EJ_RESCORE_ARGS);                 \
    else if (aligned && d <= 256) rescore_mlp_kernel<2, 2, M, true><<<g, T, 0, st>>>(EJ_RESCORE_ARGS);            \
    else if (aligned && d <= 384) rescore_mlp_kernel<3, 2, M, true><<<g, T, 0, st>>>(EJ_RESCORE_ARGS);            \
    else if (aligned && d <= 512) rescore_mlp_kernel<4, 1, M, true><<<g, T, 0, st>>>(EJ_RESCORE_ARGS);            \
    else if (aligned && d <= 768) rescore_mlp_kernel<6, 1, M, true><<<g, T, 0, st>>>(EJ_RESCORE_ARGS);            \
    else if (aligned && d <= 1024) rescore_mlp_kernel<8, 1, M, true><<<g, T, 0, st>>>(EJ_RESCORE_ARGS);           \
    else rescore_kernel<M><<<g, T, 0, st>>>(EJ_RESCORE_ARGS);
    if (mirror) {
        EJ_DISPATCH(true)
    } else {
        EJ_DISPATCH(false)
    }
#undef EJ_DISPATCH
    cudaError_t e = cudaGetLastError();
#undef EJ_RESCORE_ARGS
    if (e != cudaSuccess || fp64_band <= 0.f) return e;
    return launch_band_tier(band_list, band_count, band_cap, R, ldR, S, ldS, d, eps, out, out_cap, out_count,
                            count_only, aligned, mirror != 0, num_sms, st, bn);
}

// ---------------------------------------------------------------------------
// Panel-ordered re-score.
//
// The candidates of a clustered join reuse each row about as often as the row
// has matches (c2: ~100), but the plain re-score gathers both FP32 rows of
// every candidate from L2 (2 * 4d bytes per candidate), which makes it bound
// by L2 -> SM traffic.  Here the candidates are first bucketed (counting
// sort: histogram, scan, scatter) by (S block, R panel): a panel is P
// consecutive operand rows of R, an S block about PANEL_SBLOCK_BYTES of
// consecutive FP32 rows of S, and the buckets are processed S-block-major.  A
// CTA stages its panel's FP32 R rows in shared memory once (cp.async, 16-byte
// pieces) and gathers only the S row of each candidate from global memory, so
// the L2 -> SM bytes per candidate halve, while the CTAs running together
// work inside one S block that stays resident in L2.  Per candidate the FP32
// arithmetic, its order and the decision are those of rescore_mlp_kernel, so
// the similarities are bit-identical; only the order of the records differs.
// Buckets are cut into chunks of at most PANEL_CHUNK candidates so that one
// dense bucket does not serialise on one CTA, and CTAs take the chunks in
// bucket order from a ticket counter, so the chunks in progress at any moment
// are neighbours and their S rows stay in L2.
namespace {
constexpr int PANEL_CHUNK = 2048;
constexpr int PANEL_MAX_ROWS = 128;
constexpr int PANEL_CTAS = 3;    // CTAs per SM for rows of up to 512 values, 2 above
constexpr int SMAJ_BINS = 1024;  // a chunk whose S rows span fewer positions is described by masks per S position
// Shared memory for the staged R rows of a CTA: three CTAs per SM with the sorted chunk and the staging
// area for rows of up to 512 values, two above.
constexpr int panel_smem(int d) { return d > 512 ? 81920 : 40960; }
constexpr int64_t PANEL_SBLOCK_BYTES = 32ll << 20;
constexpr int64_t PANEL_MAX_BUCKETS = 1ll << 22;
constexpr int64_t PANEL_MIN_BUCKET = 1024;
constexpr int SCAN_THREADS = 1024;

// Bucket geometry: bucket(c) = (c.y / sb) * np + (c.x >> shift), nb = nsb * np buckets.
struct PanelGeom {
    int shift;    // log2 of the panel height P
    int64_t np;   // panels over the operand rows of R
    int64_t sb;   // operand rows of S per S block
    int64_t nsb;  // S blocks
    int64_t nb;   // buckets
};
}  // namespace

int rescore_panel_rows(int d)
{
    const int row_bytes = ((d + 3) / 4) * 16;
    int p = PANEL_MAX_ROWS;
    while (p > 8 && p * row_bytes > panel_smem(d)) p >>= 1;
    return p * row_bytes <= panel_smem(d) ? p : 0;
}

// cand_hint (0: unknown): the number of candidates.  S blocks split a panel's candidates only while a bucket
// keeps about PANEL_MIN_BUCKET of them: a sparse join is not fragmented into chunks of a few candidates, whose
// fixed cost (staging, sorting, barriers) would exceed the L2 locality gained.
static PanelGeom panel_geom(int64_t n_rows, int64_t n_rows_s, int d, uint64_t cand_hint)
{
    PanelGeom g{};
    const int P = rescore_panel_rows(d);
    while ((1 << g.shift) < P) ++g.shift;
    g.np = std::max<int64_t>(1, (n_rows + P - 1) / P);
    const int64_t row_bytes = (int64_t)((d + 3) / 4) * 16;
    const int64_t ns = std::max<int64_t>(1, n_rows_s);
    int64_t nsb = std::max<int64_t>(1, (ns * row_bytes + PANEL_SBLOCK_BYTES - 1) / PANEL_SBLOCK_BYTES);
    nsb = std::min<int64_t>(nsb, std::max<int64_t>(1, PANEL_MAX_BUCKETS / g.np));
    if (cand_hint) nsb = std::min<int64_t>(nsb, std::max<int64_t>(1, (int64_t)(cand_hint / (uint64_t)(g.np * PANEL_MIN_BUCKET))));
    g.sb = (ns + nsb - 1) / nsb;
    g.nsb = (ns + g.sb - 1) / g.sb;
    g.nb = g.nsb * g.np;
    return g;
}

__device__ __forceinline__ unsigned panel_bucket(uint2 c, int shift, int64_t np, int64_t sb)
{
    return (unsigned)((int64_t)(c.y / (uint64_t)sb) * np + (int64_t)(c.x >> shift));
}

// Bucket of a candidate in a panel geometry (single join)
struct GridBucket {
    PanelGeom g;
    __device__ __forceinline__ unsigned operator()(uint2 c) const { return panel_bucket(c, g.shift, g.np, g.sb); }
};

// Bucket of a batched candidate (a, b): its job j (the job of A row a), then the S block of b within the
// job (sb rows each), then the A row: bbase[j] + ((b - b_off[j]) / sb) nA[j] + (a - a_off[j]).  Buckets
// are ordered job by job, S block by S block, A row by A row.
struct JobBlockBucket {
    const int *row_job;
    const long long *bbase, *a_off, *b_off;
    const int *nA;
    unsigned sb;
    __device__ __forceinline__ unsigned operator()(uint2 c) const
    {
        const int j = __ldg(row_job + c.x);
        const unsigned blk = (unsigned)((long long)c.y - __ldg(b_off + j)) / sb;
        return (unsigned)(__ldg(bbase + j) + (long long)blk * __ldg(nA + j) + ((long long)c.x - __ldg(a_off + j)));
    }
};

// cnt[bucket(c)] += 1 for every candidate (one atomic per group of lanes sharing a bucket)
template <class Bucket>
__global__ void __launch_bounds__(256) panel_hist_kernel(const uint2 *__restrict__ cand,
                                                         const unsigned long long *__restrict__ cand_count,
                                                         uint64_t cand_cap, Bucket bucket, unsigned long long *cnt)
{
    const int lane = threadIdx.x & 31;
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = w0 * 32; base < n; base += nw * 32) {
        const uint64_t k = base + lane;
        const bool ok = k < n;
        const unsigned p = ok ? bucket(cand[k]) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, p);
        if (ok && lane == __ffs(peers) - 1) atomicAdd(cnt + p, (unsigned long long)__popc(peers));
    }
}

// Scan of the bucket counts in three phases (SCAN_ITEMS buckets per block): per-block totals of cnt and of
// the chunk counts ceil(cnt / PANEL_CHUNK); one block scans those totals; each block then writes
// off[b] = sum of cnt[< b], cursor[b] = off[b] and choff[b] = sum of the chunk counts of the buckets < b
// (off[nb] = candidates, choff[nb] = chunks).
constexpr int SCAN_ITEMS = SCAN_THREADS * 8;

// Block-wide inclusive scan of two values per thread (x, y); returns the block totals through tx, ty.
__device__ __forceinline__ void block_scan2(unsigned long long &x, unsigned long long &y, unsigned long long &tx,
                                            unsigned long long &ty)
{
    __shared__ unsigned long long wa[32], wb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long ya = __shfl_up_sync(0xffffffffu, x, o);
        const unsigned long long yb = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) {
            x += ya;
            y += yb;
        }
    }
    if (lane == 31) {
        wa[warp] = x;
        wb[warp] = y;
    }
    __syncthreads();
    if (warp == 0) {
        unsigned long long a = lane < (int)(blockDim.x >> 5) ? wa[lane] : 0ull;
        unsigned long long b = lane < (int)(blockDim.x >> 5) ? wb[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long ya = __shfl_up_sync(0xffffffffu, a, o);
            const unsigned long long yb = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) {
                a += ya;
                b += yb;
            }
        }
        wa[lane] = a;
        wb[lane] = b;
    }
    __syncthreads();
    if (warp) {
        x += wa[warp - 1];
        y += wb[warp - 1];
    }
    tx = wa[(blockDim.x >> 5) - 1];
    ty = wb[(blockDim.x >> 5) - 1];
    __syncthreads();
}

__global__ void __launch_bounds__(SCAN_THREADS) panel_scan_reduce_kernel(const unsigned long long *__restrict__ cnt,
                                                                         int64_t nb, unsigned long long *tot)
{
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_ITEMS;
    unsigned long long a = 0, c = 0;
    for (int k = threadIdx.x; k < SCAN_ITEMS; k += SCAN_THREADS) {
        const int64_t i = b0 + k;
        const unsigned long long v = i < nb ? cnt[i] : 0ull;
        a += v;
        c += (v + PANEL_CHUNK - 1) / PANEL_CHUNK;
    }
    unsigned long long ta, tc;
    block_scan2(a, c, ta, tc);
    if (threadIdx.x == 0) {
        tot[2 * blockIdx.x] = ta;
        tot[2 * blockIdx.x + 1] = tc;
    }
}

// one block: exclusive scan of the per-block totals in place (tot[2 * blocks], tot[2 * blocks + 1] = totals)
__global__ void __launch_bounds__(SCAN_THREADS) panel_scan_top_kernel(unsigned long long *tot, int blocks)
{
    __shared__ unsigned long long carry_a, carry_c;
    if (threadIdx.x == 0) carry_a = carry_c = 0ull;
    __syncthreads();
    for (int base = 0; base < blocks; base += SCAN_THREADS) {
        const int i = base + threadIdx.x;
        const unsigned long long va = i < blocks ? tot[2 * i] : 0ull, vc = i < blocks ? tot[2 * i + 1] : 0ull;
        unsigned long long a = va, c = vc, ta, tc;
        block_scan2(a, c, ta, tc);
        if (i < blocks) {
            tot[2 * i] = carry_a + a - va;
            tot[2 * i + 1] = carry_c + c - vc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_a += ta;
            carry_c += tc;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tot[2 * blocks] = carry_a;
        tot[2 * blocks + 1] = carry_c;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) panel_scan_down_kernel(const unsigned long long *__restrict__ cnt,
                                                                       int64_t nb, const unsigned long long *tot,
                                                                       unsigned long long *off,
                                                                       unsigned long long *cursor,
                                                                       unsigned long long *choff)
{
    // each thread scans 8 consecutive buckets of the block's SCAN_ITEMS
    constexpr int PER = SCAN_ITEMS / SCAN_THREADS;
    const int64_t i0 = (int64_t)blockIdx.x * SCAN_ITEMS + (int64_t)threadIdx.x * PER;
    unsigned long long v[PER], a = 0, c = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = i0 + k < nb ? cnt[i0 + k] : 0ull;
        a += v[k];
        c += (v[k] + PANEL_CHUNK - 1) / PANEL_CHUNK;
    }
    unsigned long long ta, tc;
    const unsigned long long a_in = a, c_in = c;
    block_scan2(a, c, ta, tc);
    unsigned long long ea = tot[2 * blockIdx.x] + a - a_in, ec = tot[2 * blockIdx.x + 1] + c - c_in;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (i0 + k < nb) {
            off[i0 + k] = ea;
            cursor[i0 + k] = ea;
            choff[i0 + k] = ec;
        }
        ea += v[k];
        ec += (v[k] + PANEL_CHUNK - 1) / PANEL_CHUNK;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        off[nb] = tot[2 * gridDim.x];
        choff[nb] = tot[2 * gridDim.x + 1];
    }
}

// sorted[cursor[b]++] = candidate, b its bucket (one atomic per group of lanes sharing a bucket)
template <class Bucket>
__global__ void __launch_bounds__(256) panel_scatter_kernel(const uint2 *__restrict__ cand,
                                                            const unsigned long long *__restrict__ cand_count,
                                                            uint64_t cand_cap, Bucket bucket,
                                                            unsigned long long *cursor, uint2 *__restrict__ sorted)
{
    const int lane = threadIdx.x & 31;
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = w0 * 32; base < n; base += nw * 32) {
        const uint64_t k = base + lane;
        const bool ok = k < n;
        const uint2 c = ok ? cand[k] : make_uint2(0u, 0u);
        const unsigned p = ok ? bucket(c) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, p);
        const int leader = __ffs(peers) - 1;
        unsigned long long pos = 0;
        if (ok && lane == leader) pos = atomicAdd(cursor + p, (unsigned long long)__popc(peers));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (ok) sorted[pos + __popc(peers & ((1u << lane) - 1u))] = c;
    }
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Sum over the 32 lanes of C values per lane at once (transposed butterfly): at each of the first
// log2(C) levels a lane keeps half of its values, hands the other half to its partner and adds the
// partner's half of its own; the remaining levels are the plain butterfly on the one value left.  Every
// value is combined over the same lane pairs (lane, lane ^ o), o = 16, 8, 4, 2, 1, as in
// `v += __shfl_xor_sync(v, o)`, so each total is bit-identical to that butterfly, for
// log2(C) + 5 - ... shuffles in place of 5 C.  On return lane c * (32 / C) holds the total of value c.
template <int C>
__device__ __forceinline__ float transpose_sum(float (&p)[C], int lane)
{
    float v[C];
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = p[k];
    int n = C;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (n > 1) {
            const bool hi = lane & o;
            const int h = n >> 1;
#pragma unroll
            for (int k = 0; k < C / 2; ++k) {
                if (k < h) {
                    const float send = hi ? v[k] : v[k + h];
                    const float keep = hi ? v[k + h] : v[k];
                    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            n = h;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
    return v[0];
}

// Per-warp staged emission of re-score results: each warp collects its records in a shared-memory
// staging area of PANEL_STG records and claims global space with one atomic per flush, so no block-wide
// barrier is needed per step.  mirror: a pair (i, j), i != j, is written as (i, j) and (j, i).
constexpr int PANEL_STG = 96;
__device__ __forceinline__ ejoin_pair swapped(const ejoin_pair &r) { return ejoin_pair{r.j, r.i, r.sim}; }
__device__ __forceinline__ BatchPair swapped(const BatchPair &r) { return BatchPair{r.job, r.j, r.i, r.sim}; }
template <bool MIRROR, typename Rec>
__device__ __forceinline__ void warp_emit_rec(bool emit, const Rec &rec, Rec *stg, int &stg_n,
                                              unsigned long long *out_count, Rec *__restrict__ out, uint64_t out_cap,
                                              int count_only, int lane, bool final_flush)
{
    const int mine = emit ? ((MIRROR && rec.i != rec.j) ? 2 : 1) : 0;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    if (stg_n + tot > PANEL_STG || (final_flush && stg_n + tot > 0)) {
        // flush what is staged, then this step's records go straight to global memory
        const int n_all = stg_n + tot;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(out_count, (unsigned long long)n_all);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (!count_only) {
            __syncwarp();
            for (int x = lane; x < stg_n; x += 32)
                if (base + (unsigned long long)x < out_cap) out[base + x] = stg[x];
            if (mine) {
                const unsigned long long pos = base + (unsigned long long)(stg_n + incl - mine);
                if (pos < out_cap) out[pos] = rec;
                if (mine == 2 && pos + 1 < out_cap) out[pos + 1] = swapped(rec);
            }
        }
        stg_n = 0;
        __syncwarp();
        return;
    }
    if (mine && !count_only) {
        const int pos = stg_n + incl - mine;
        stg[pos] = rec;
        if (mine == 2) stg[pos + 1] = swapped(rec);
    }
    stg_n += tot;
    __syncwarp();
}

template <bool MIRROR>
__device__ __forceinline__ void warp_emit(bool emit, uint32_t i, uint32_t j, float sim, ejoin_pair *stg, int &stg_n,
                                          unsigned long long *out_count, ejoin_pair *__restrict__ out,
                                          uint64_t out_cap, int count_only, int lane, bool final_flush)
{
    warp_emit_rec<MIRROR>(emit, ejoin_pair{i, j, sim}, stg, stg_n, out_count, out, out_cap, count_only, lane,
                          final_flush);
}

// A chunk whose S rows span few positions (rescore_panel_kernel, clustered rows in sketch order), given as
// one mask per S position of the panel rows it pairs with (P <= 32).  Each warp takes two S positions at a
// time and holds both S rows in registers; every panel row either of them pairs with is read from shared
// memory once and serves both, so a dense block of candidates reads half an R row per candidate.  Each
// result is kept by one lane until 32 are decided and emitted together (the band-list entries of the 32
// claimed with one atomic).  Lane partials, their order and the reduction tree are those of
// rescore_mlp_kernel (fmaf(R element, S element, acc) over v, then the butterfly pairs), so the similarities
// are bit-identical to the R-major path.
template <int V, bool MIRROR>
__device__ __forceinline__ void rescore_smajor_masked(
    const unsigned *masks, int nbins, unsigned s_lo, long long row0, const float4 *panel, int d4,
    const float *__restrict__ S, int64_t ldS, const uint32_t *__restrict__ idsR, const uint32_t *__restrict__ idsS,
    const float *__restrict__ invR, const float *__restrict__ invS, float eps, float fp64_band,
    unsigned long long *band_count, uint2 *__restrict__ band_list, uint64_t band_cap, ejoin_pair *stg, int &stg_n,
    unsigned long long *out_count, ejoin_pair *__restrict__ out, uint64_t out_cap, int count_only, int lane, int warp)
{
    // candidate k of the current batch of up to 32 is kept by lane k (its dot product, panel row and S
    // position); the batch is decided and emitted by all lanes at once
    int nb = 0;  // warp-uniform
    float my_dot = 0.f;
    uint32_t my_r = 0, my_p = 0;
    auto flush = [&]() {
        bool my_emit = false, near = false;
        uint32_t gi = 0, gj = 0;
        float sim = 0.f;
        if (lane < nb) {
            const long long o = row0 + my_r;
            const uint32_t sidx = s_lo + my_p;
            gi = idsR ? idsR[o] : (uint32_t)o;
            gj = idsS ? idsS[sidx] : sidx;
            sim = fminf(1.f, fmaxf(-1.f, my_dot * (invR[o] * invS[sidx])));
            near = fabsf(sim - eps) < fp64_band;  // near eps: decided by the accurate tier
            my_emit = sim >= eps && !near;
        }
        // the batch's entries of the band list claimed with one atomic
        const unsigned nmask = __ballot_sync(0xffffffffu, near);
        if (nmask) {  // warp-uniform
            const int leader = __ffs(nmask) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(band_count, (unsigned long long)__popc(nmask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (near) {
                const unsigned long long q = base + (unsigned long long)__popc(nmask & ((1u << lane) - 1u));
                if (q < band_cap) band_list[q] = make_uint2(gi, gj);
            }
        }
        warp_emit<MIRROR>(my_emit, gi, gj, sim, stg, stg_n, out_count, out, out_cap, count_only, lane, false);
        nb = 0;
    };
    auto keep = [&](float dot, uint32_t r, uint32_t p) {
        if (lane == nb) {
            my_dot = dot;
            my_r = r;
            my_p = p;
        }
        ++nb;
    };
    auto load_s = [&](float4 (&b)[V], uint32_t p) {
        const uint32_t sidx = s_lo + p;
        const uint32_t j = idsS ? idsS[sidx] : sidx;
        const float4 *g = reinterpret_cast<const float4 *>(S + (int64_t)j * ldS);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int x = lane + 32 * v;
            b[v] = x < d4 ? __ldg(g + x) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto dot_with = [&](const float4 (&a)[V], const float4 (&b)[V]) {
        float acc = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            acc = fmaf(a[v].x, b[v].x, acc);
            acc = fmaf(a[v].y, b[v].y, acc);
            acc = fmaf(a[v].z, b[v].z, acc);
            acc = fmaf(a[v].w, b[v].w, acc);
        }
        return acc;
    };
    for (int p0 = 2 * warp; p0 < nbins; p0 += 2 * RS_WARPS) {
        const unsigned m0 = masks[p0];
        const unsigned m1 = p0 + 1 < nbins ? masks[p0 + 1] : 0u;
        if ((m0 | m1) == 0u) continue;  // warp-uniform
        float4 b0[V], b1[V];
#pragma unroll
        for (int v = 0; v < V; ++v) b0[v] = b1[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m0) load_s(b0, (uint32_t)p0);
        if (m1) load_s(b1, (uint32_t)p0 + 1u);
        unsigned m = m0 | m1;
        while (m) {  // warp-uniform
            const int r = __ffs(m) - 1;
            m &= m - 1u;
            if (nb > 30) flush();
            float4 a[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int x = lane + 32 * v;
                a[v] = x < d4 ? panel[(uint32_t)r * (uint32_t)d4 + x] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const bool in0 = (m0 >> r) & 1u, in1 = (m1 >> r) & 1u;
            if (in0 && in1) {
                // both positions pair with row r: one transposed reduction of the two partials
                float part[2] = {dot_with(a, b0), dot_with(a, b1)};
                const float tot = transpose_sum<2>(part, lane);
                const float t0 = __shfl_sync(0xffffffffu, tot, 0), t1 = __shfl_sync(0xffffffffu, tot, 16);
                keep(t0, (uint32_t)r, (uint32_t)p0);
                keep(t1, (uint32_t)r, (uint32_t)p0 + 1u);
            } else {
                float acc = in0 ? dot_with(a, b0) : dot_with(a, b1);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                keep(acc, (uint32_t)r, in0 ? (uint32_t)p0 : (uint32_t)p0 + 1u);
            }
        }
    }
    if (nb > 0) flush();
}

template <int V, int C, bool MIRROR, int CTAS>
__global__ void __launch_bounds__(RS_WARPS * 32, CTAS) rescore_panel_kernel(
    const uint2 *__restrict__ sorted, const unsigned long long *__restrict__ off,
    const unsigned long long *__restrict__ choff, PanelGeom pg, const long long *__restrict__ nA_dev,
    const float *__restrict__ R, int64_t ldR, const float *__restrict__ S, int64_t ldS, int d,
    const uint32_t *__restrict__ idsR, const uint32_t *__restrict__ idsS, const float *__restrict__ invR,
    const float *__restrict__ invS, float eps, float fp64_band, ejoin_pair *__restrict__ out, uint64_t out_cap,
    unsigned long long *out_count, unsigned long long *band_count, int count_only, uint2 *__restrict__ band_list,
    uint64_t band_cap, unsigned long long *chunk_ticket)
{
    static_assert(RS_PER_WARP % C == 0 && (C & (C - 1)) == 0, "candidates per warp step");
    extern __shared__ float4 dyn[];
    __shared__ unsigned long long s_tk[2];  // chunk tickets: this chunk's successor, double-buffered
    // counts of the chunk's counting sort: R rows, or (rows of more than 512 values) S positions
    __shared__ int rcnt[V >= 6 ? SMAJ_BINS : PANEL_MAX_ROWS];
    __shared__ unsigned char rused[PANEL_MAX_ROWS];  // the panel rows the chunk uses (only those are staged)
    __shared__ unsigned s_range[2];  // the chunk's smallest and largest S operand row
    __shared__ ejoin_pair stg_all[RS_WARPS][PANEL_STG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ejoin_pair *stg = stg_all[warp];
    int stg_n = 0;
    const int d4 = d >> 2;
    const int shift = pg.shift;
    const int P = 1 << shift;
    float4 *panel = dyn;                                                // P x d4
    uint2 *cs = reinterpret_cast<uint2 *>(dyn + (size_t)P * (size_t)d4);  // the chunk, sorted by row
    const long long nA = *nA_dev;
    const unsigned long long n_chunks = choff[pg.nb];
    // chunks are handed out in order from one ticket counter, so the chunks in progress at any moment are
    // neighbours in bucket order (their S rows stay in L2); the successor's ticket is taken one chunk ahead
    if (threadIdx.x == 0) s_tk[1] = atomicAdd(chunk_ticket, 1ull);
    __syncthreads();
    int par = 0;
    for (unsigned long long ch = s_tk[1]; ch < n_chunks; ch = s_tk[par], par ^= 1) {
        if (threadIdx.x == 0) s_tk[par] = atomicAdd(chunk_ticket, 1ull);  // read after this chunk's barriers
        // the chunk's bucket: the last b with choff[b] <= ch (it holds at least one chunk)
        int64_t lo = 0, hi = pg.nb;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(choff + mid) <= ch) lo = mid;
            else hi = mid;
        }
        const unsigned long long k0 = __ldg(off + lo) + (ch - __ldg(choff + lo)) * (unsigned long long)PANEL_CHUNK;
        const int len = (int)min((unsigned long long)PANEL_CHUNK, __ldg(off + lo + 1) - k0);
        const long long row0 = (long long)(lo % pg.np) << shift;  // the bucket's R panel
        const int rows = (int)min((long long)P, nA - row0);
        __syncthreads();  // the previous chunk is done with the panel, the sorted chunk and the counts
        // the span of the chunk's S rows: within SMAJ_BINS positions (clustered rows in sketch order), the
        // chunk is sorted by S row and each S row is gathered once for all its candidates; otherwise by R row
        // the chunk's candidates, read once into registers (PANEL_CHUNK / blockDim.x per thread)
        constexpr int ITEMS = PANEL_CHUNK / (RS_WARPS * 32);
        uint2 mine[ITEMS];
#pragma unroll
        for (int t = 0; t < ITEMS; ++t) {
            const int k = threadIdx.x + t * (RS_WARPS * 32);
            mine[t] = k < len ? sorted[k0 + k] : make_uint2(0u, 0u);
        }
        bool smajor = false;
        unsigned s_lo = 0;
        if constexpr (V >= 6) {
            // rows of more than 512 values: when the chunk's S rows span fewer than SMAJ_BINS positions
            // (clustered rows in sketch order) it is sorted by S row and each S row is gathered once for all
            // its candidates (rows of up to 512 values keep their registers for the R-major path)
            if (threadIdx.x == 0) {
                s_range[0] = 0xffffffffu;
                s_range[1] = 0u;
            }
            __syncthreads();
            unsigned lo = 0xffffffffu, hi = 0u;
#pragma unroll
            for (int t = 0; t < ITEMS; ++t) {
                if (threadIdx.x + t * (RS_WARPS * 32) < len) {
                    lo = min(lo, mine[t].y);
                    hi = max(hi, mine[t].y);
                }
            }
            lo = __reduce_min_sync(0xffffffffu, lo);
            hi = __reduce_max_sync(0xffffffffu, hi);
            if (lane == 0) {
                atomicMin(&s_range[0], lo);
                atomicMax(&s_range[1], hi);
            }
            __syncthreads();
            s_lo = s_range[0];
            smajor = s_range[1] - s_lo < (unsigned)SMAJ_BINS && P <= 32;  // one 32-bit row mask per position
        }
        // counting sort of the chunk (S-major: one mask of panel rows per S position instead); the R rows it
        // uses are flagged and only those are staged (the copies are in flight during the scan and the scatter)
        const int nbins = smajor ? (int)(s_range[1] - s_lo) + 1 : P;
        for (int r = threadIdx.x; r < nbins; r += blockDim.x) rcnt[r] = 0;
        for (int r = threadIdx.x; r < P; r += blockDim.x) rused[r] = 0;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < ITEMS; ++t) {
            if (threadIdx.x + t * (RS_WARPS * 32) < len) {
                if (smajor)
                    atomicOr(reinterpret_cast<unsigned *>(&rcnt[(int)(mine[t].y - s_lo)]), 1u << (mine[t].x - row0));
                else
                    atomicAdd(&rcnt[(int)(mine[t].x - row0)], 1);
                rused[mine[t].x - row0] = 1;
            }
        }
        __syncthreads();
        for (int r = warp; r < rows; r += RS_WARPS) {
            if (!rused[r]) continue;  // warp-uniform
            const long long o = row0 + r;
            const uint32_t src = idsR ? idsR[o] : (uint32_t)o;
            const float4 *g = reinterpret_cast<const float4 *>(R + (int64_t)src * ldR);
            for (int x = lane; x < d4; x += 32) cp_async16(panel + r * d4 + x, g + x);
        }
        if (V >= 6 && smajor) {
            // the masks are the chunk's whole description: no scan and no scatter
        } else if (warp == 0) {
            // exclusive scan of the P <= 128 counts, 4 per lane
            int v[PANEL_MAX_ROWS / 32], s = 0;
#pragma unroll
            for (int t = 0; t < PANEL_MAX_ROWS / 32; ++t) {
                const int r = lane * (PANEL_MAX_ROWS / 32) + t;
                v[t] = r < P ? rcnt[r] : 0;
                s += v[t];
            }
            int incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int run = incl - s;
#pragma unroll
            for (int t = 0; t < PANEL_MAX_ROWS / 32; ++t) {
                const int r = lane * (PANEL_MAX_ROWS / 32) + t;
                if (r < P) rcnt[r] = run;
                run += v[t];
            }
        }
        __syncthreads();
        if (!smajor) {
#pragma unroll
            for (int t = 0; t < ITEMS; ++t)
                if (threadIdx.x + t * (RS_WARPS * 32) < len) cs[atomicAdd(&rcnt[(int)(mine[t].x - row0)], 1)] = mine[t];
        }
        cp_async_wait_all();
        __syncthreads();
        if constexpr (V >= 6) {
            if (smajor) {
                rescore_smajor_masked<V, MIRROR>(reinterpret_cast<const unsigned *>(rcnt), nbins, s_lo, row0, panel,
                                                 d4, S, ldS, idsR, idsS, invR, invS, eps, fp64_band, band_count,
                                                 band_list, band_cap, stg, stg_n, out_count, out, out_cap, count_only,
                                                 lane, warp);
                continue;
            }
        }
        // warps take the chunk's candidates 16 at a time, with no block-wide step
        for (int gbase = warp * RS_PER_WARP; gbase < len; gbase += RS_PER_BLOCK) {
            bool my_emit = false;
            uint32_t my_i = 0, my_j = 0;
            float my_sim = 0.f;
            // lanes 0..15 fetch the warp's 16 candidates, their original ids, scales and panel rows
            uint32_t gi = 0, gj = 0, lr = 0;
            float sc = 0.f;
            bool valid = false;
            if (lane < RS_PER_WARP && gbase + lane < len) {
                const uint2 c = cs[gbase + lane];
                gi = idsR ? idsR[c.x] : c.x;
                gj = idsS ? idsS[c.y] : c.y;
                lr = (uint32_t)((long long)c.x - row0);
                sc = invR[c.x] * invS[c.y];
                valid = true;
            }
            const unsigned vmask = __ballot_sync(0xffffffffu, valid);
            if (vmask) {  // warp-uniform
                float4 a[V];
                uint32_t cur = 0xffffffffu;  // panel row held in a[]
#pragma unroll
                for (int v = 0; v < V; ++v) a[v] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
                for (int q0 = 0; q0 < RS_PER_WARP; q0 += C) {
                    if (!((vmask >> q0) & 1u)) break;  // warp-uniform
                    float4 b[C][V];
                    uint32_t rr[C];
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const uint32_t jj = __shfl_sync(0xffffffffu, gj, q0 + c);
                        rr[c] = __shfl_sync(0xffffffffu, lr, q0 + c);
                        const bool ok = (vmask >> (q0 + c)) & 1u;
                        const float4 *srow = reinterpret_cast<const float4 *>(S + (int64_t)jj * ldS);
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const int g = lane + 32 * v;
                            b[c][v] = ok && g < d4 ? __ldg(srow + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                    // all C * V gathers in flight together (see rescore_mlp_kernel)
                    asm volatile("membar.cta;" ::: "memory");
                    float part[C];
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const bool ok = (vmask >> (q0 + c)) & 1u;
                        if (ok && rr[c] != cur) {  // warp-uniform; rare, the chunk is sorted by row
                            cur = rr[c];
#pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const int g = lane + 32 * v;
                                a[v] = g < d4 ? panel[cur * (uint32_t)d4 + g] : make_float4(0.f, 0.f, 0.f, 0.f);
                            }
                        }
                        float acc = 0.f;
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            acc = fmaf(a[v].x, b[c][v].x, acc);
                            acc = fmaf(a[v].y, b[c][v].y, acc);
                            acc = fmaf(a[v].z, b[c][v].z, acc);
                            acc = fmaf(a[v].w, b[c][v].w, acc);
                        }
                        part[c] = acc;
                    }
                    const float tot = transpose_sum<C>(part, lane);
                    // lane q0 + c takes candidate c's dot product from lane c * (32 / C) and decides it
                    const float mine = __shfl_sync(0xffffffffu, tot, ((lane - q0) & (C - 1)) * (32 / C));
                    if (lane >= q0 && lane < q0 + C && ((vmask >> lane) & 1u)) {
                        float sim = mine * sc;
                        sim = fminf(1.f, fmaxf(-1.f, sim));
                        bool emit = sim >= eps;
                        if (fabsf(sim - eps) < fp64_band) {
                            // near eps: decided by the accurate tier (rescore_band_kernel)
                            const unsigned long long p = atomicAdd(band_count, 1ull);
                            if (p < band_cap) band_list[p] = make_uint2(gi, gj);
                            emit = false;
                        }
                        my_emit = emit;
                        my_i = gi;
                        my_j = gj;
                        my_sim = sim;
                    }
                }
            }
            warp_emit<MIRROR>(my_emit, my_i, my_j, my_sim, stg, stg_n, out_count, out, out_cap, count_only, lane,
                              false);
        }
    }
    warp_emit<MIRROR>(false, 0u, 0u, 0.f, stg, stg_n, out_count, out, out_cap, count_only, lane, true);
}

size_t rescore_panel_buf_bytes(int64_t n_rows, int64_t n_rows_s, int d, uint64_t cand_hint)
{
    if (rescore_panel_rows(d) == 0) return 0;
    const PanelGeom g = panel_geom(n_rows, n_rows_s, d, cand_hint);
    const int64_t scan_blocks = (g.nb + SCAN_ITEMS - 1) / SCAN_ITEMS;
    return (size_t)(4 * g.nb + 2 + 2 * scan_blocks + 2 + 2) * sizeof(unsigned long long);
}

template <int V, int C, bool M, int CTAS = PANEL_CTAS>
static cudaError_t launch_panel_kernel(unsigned grid, int num_sms, size_t smem, cudaStream_t st, const uint2 *sorted,
                                       const unsigned long long *off, const unsigned long long *choff,
                                       const PanelGeom &pg, const long long *nA_dev, const float *R, int64_t ldR,
                                       const float *S, int64_t ldS, int d, const uint32_t *idsR,
                                       const uint32_t *idsS, const float *invR, const float *invS, float eps,
                                       float fp64_band, ejoin_pair *out, uint64_t out_cap,
                                       unsigned long long *out_count, unsigned long long *band_count, int count_only,
                                       uint2 *band_list, uint64_t band_cap, unsigned long long *chunk_ticket)
{
    // the shared-memory opt-in, once per device and instantiation
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!((configured >> dev) & 1ull)) {
        e = cudaFuncSetAttribute(rescore_panel_kernel<V, C, M, CTAS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 panel_smem(CTAS == PANEL_CTAS ? 512 : 1024) + PANEL_CHUNK * (int)sizeof(uint2));
        if (e != cudaSuccess) return e;
        configured |= 1ull << dev;
    }
    // persistent CTAs: no more than are resident at once (a later wave would start after the first finished)
    grid = std::min<unsigned>(grid, (unsigned)(num_sms * CTAS));
    rescore_panel_kernel<V, C, M, CTAS><<<grid, RS_WARPS * 32, smem, st>>>(
        sorted, off, choff, pg, nA_dev, R, ldR, S, ldS, d, idsR, idsS, invR, invS, eps, fp64_band, out, out_cap,
        out_count, band_count, count_only, band_list, band_cap, chunk_ticket);
    return cudaGetLastError();
}

cudaError_t launch_rescore_panels(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                  uint2 *sorted, void *panel_buf, int64_t n_rows, int64_t n_rows_s,
                                  uint64_t cand_hint, const long long *nA_dev, const float *R, int64_t ldR, const float *S, int64_t ldS,
                                  int d, const uint32_t *idsR, const uint32_t *idsS, const float *invR,
                                  const float *invS, float eps, float fp64_band, ejoin_pair *out, uint64_t out_cap,
                                  unsigned long long *out_count, unsigned long long *band_count, int count_only,
                                  int num_sms, cudaStream_t st, uint2 *band_list, uint64_t band_cap, int mirror,
                                  const BandNorms *bn)
{
    if (cand_cap == 0) return cudaSuccess;
    if (fp64_band > 0.f && (!band_list || band_cap < cand_cap)) return cudaErrorInvalidValue;
    const bool aligned = (d % 4 == 0) && (ldR % 4 == 0) && (ldS % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(R) % 16 == 0) && (reinterpret_cast<uintptr_t>(S) % 16 == 0);
    const int P = rescore_panel_rows(d);
    if (!aligned || d > 1024 || P == 0 || !sorted || !panel_buf) return cudaErrorInvalidValue;
    const PanelGeom g = panel_geom(n_rows, n_rows_s, d, cand_hint);
    if (g.nb >= (int64_t)0xffffffffll) return cudaErrorInvalidValue;
    unsigned long long *cnt = static_cast<unsigned long long *>(panel_buf);
    unsigned long long *off = cnt + g.nb;        // nb + 1
    unsigned long long *cursor = off + g.nb + 1;  // nb
    unsigned long long *choff = cursor + g.nb;    // nb + 1
    unsigned long long *tot = choff + g.nb + 1;    // 2 * scan_blocks + 2
    const int64_t scan_blocks = (g.nb + SCAN_ITEMS - 1) / SCAN_ITEMS;
    unsigned long long *chunk_ticket = tot + 2 * scan_blocks + 2;  // 2 (one used)
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)g.nb * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(chunk_ticket, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    const unsigned gs = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((cand_cap + 255) / 256, (uint64_t)num_sms * 8));
    panel_hist_kernel<<<gs, 256, 0, st>>>(cand, cand_count, cand_cap, GridBucket{g}, cnt);
    panel_scan_reduce_kernel<<<(unsigned)scan_blocks, SCAN_THREADS, 0, st>>>(cnt, g.nb, tot);
    panel_scan_top_kernel<<<1, SCAN_THREADS, 0, st>>>(tot, (int)scan_blocks);
    panel_scan_down_kernel<<<(unsigned)scan_blocks, SCAN_THREADS, 0, st>>>(cnt, g.nb, tot, off, cursor, choff);
    panel_scatter_kernel<<<gs, 256, 0, st>>>(cand, cand_count, cand_cap, GridBucket{g}, cursor, sorted);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const uint64_t max_chunks = (uint64_t)g.nb + cand_cap / PANEL_CHUNK + 1;
    const unsigned grid =
        (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(max_chunks, (uint64_t)num_sms * PANEL_CTAS));
    const size_t smem = (size_t)P * (size_t)(d / 4) * 16 + PANEL_CHUNK * sizeof(uint2);
#define EJ_PANEL_ARGS                                                                                            \
    grid, num_sms, smem, st, sorted, off, choff, g, nA_dev, R, ldR, S, ldS, d, idsR, idsS, invR, invS, eps, fp64_band, out, \
        out_cap, out_count, band_count, count_only, band_list, band_cap, chunk_ticket
#define EJ_PANEL(M)                                                                            \
    if (d <= 128) e = launch_panel_kernel<1, 8, M>(EJ_PANEL_ARGS);                             \
    else if (d <= 256) e = launch_panel_kernel<2, 4, M>(EJ_PANEL_ARGS);                        \
    else if (d <= 384) e = launch_panel_kernel<3, 4, M>(EJ_PANEL_ARGS);                        \
    else if (d <= 512) e = launch_panel_kernel<4, 2, M>(EJ_PANEL_ARGS);                        \
    else if (d <= 768) e = launch_panel_kernel<6, 2, M, 2>(EJ_PANEL_ARGS);                     \
    else e = launch_panel_kernel<8, 1, M, 2>(EJ_PANEL_ARGS);
    if (mirror) {
        EJ_PANEL(true)
    } else {
        EJ_PANEL(false)
    }
#undef EJ_PANEL
#undef EJ_PANEL_ARGS
    if (e != cudaSuccess || fp64_band <= 0.f) return e;
    return launch_band_tier(band_list, band_count, band_cap, R, ldR, S, ldS, d, eps, out, out_cap, out_count,
                            count_only, true, mirror != 0, num_sms, st, bn);
}

// job of the first row of every panel of 2^shift rows: the last j with a_off[j] <= p 2^shift
__global__ void __launch_bounds__(256) panel_job_kernel(const long long *__restrict__ a_off, int n_jobs, int shift,
                                                        int64_t np, int *__restrict__ panel_job)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const long long r = (long long)p << shift;
    int lo = 0, hi = n_jobs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a_off + mid) <= r) lo = mid;
        else hi = mid;
    }
    panel_job[p] = lo;
}

// Streaming batched re-score.  The candidates are counting-sorted by A row (one bucket per concatenated A
// row), so each A row's candidates are contiguous; the A row then stays in registers for its whole run.
// Every warp walks its own units of 32 consecutive sorted candidates with no block-wide barrier: the S row
// of each candidate is copied into a per-warp shared-memory ring of NS slots (cp.async, NS - 1 rows in
// flight while one is consumed), and the next unit's candidate, job and scale lookups are issued in
// stages across the current unit's steps.  A slot holds 32 V float4 (positions past the row's end stay
// zero), and lanes with no candidate (the stream's tail) repeat a valid one, so the per-candidate path
// has no branch.  Lane partials, their order, the reduction tree, the clamp and the decision are
// those of rescore_batch_kernel, so the records are identical.
template <int V, int C, int NS, bool RAGGED, int CTAS>
__global__ void __launch_bounds__(RS_WARPS * 32, CTAS) rescore_stream_batch_kernel(
    const uint2 *__restrict__ sorted, const unsigned long long *__restrict__ cand_count, uint64_t cand_cap,
    const int *__restrict__ row_job, const BatchRows br, int d, const float *__restrict__ invA,
    const float *__restrict__ invB, float fp64_band, BatchPair *__restrict__ out, uint64_t out_cap,
    unsigned long long *out_count, unsigned long long *band_count, unsigned long long *unit_ticket)
{
    static_assert((C & (C - 1)) == 0 && 32 % C == 0 && NS >= 2 && NS <= 8, "step shape");
    constexpr int STEPS = 32 / C;
    // the first step that issues a copy for the next unit, and the stages of its lookups before it
    constexpr int FIN = (33 - NS) / C;
    constexpr int R2 = FIN / 3, R3 = (2 * FIN) / 3;
    static_assert(FIN >= 2 && R2 >= 1 && R3 > R2 && FIN > R3, "lookup stages");
    constexpr int SLOT = 32 * V;  // float4 per ring slot
    extern __shared__ float4 dyn[];
    __shared__ BatchPair stg_all[RS_WARPS][PANEL_STG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d4 = d >> 2;
    float4 *ring = dyn + (size_t)warp * NS * SLOT;
    BatchPair *stg = stg_all[warp];
    int stg_n = 0;
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    const uint64_t units = (n + 31) / 32;
    // units are handed out in order from one ticket counter, so the units in progress at any moment are
    // consecutive (the S rows they read stay in L2); each warp holds the ticket of its next unit
    auto ticket = [&]() {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(unit_ticket, 1ull);
        return (uint64_t)__shfl_sync(0xffffffffu, t, 0);
    };
    uint64_t u = ticket();
    if (u >= units) return;  // warp-uniform; the kernel has no block-wide barrier
    uint64_t un = ticket();

    // this lane's candidate of the current unit (lanes past the end repeat the unit's first)
    uint32_t x, job, gi, gj;
    const float *sp;
    float sc, ej;
    bool ok;
    {
        const uint64_t k = u * 32 + lane;
        ok = k < n;
        const uint2 c = sorted[ok ? k : u * 32];
        job = (uint32_t)__ldg(row_job + c.x);
        x = c.x;
        gi = batch_row_a(br, c.x, job);
        gj = batch_row_b(br, c.y, job);
        sp = br.S[job] + (int64_t)gj * br.ldS[job];
        sc = invA[c.x] * invB[c.y];
        ej = __ldg(br.eps + job);
    }
    const uint32_t ring_s = smem_u32(ring) + (uint32_t)lane * 16u;
    // ragged rows: the slot positions past the row's end are zeroed once and never copied to
    if (RAGGED) {
        for (int t = lane; t < NS * SLOT; t += 32)
            if (t % SLOT >= d4) ring[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
    }
    auto issue = [&](const float *row, int slot) {
        const float4 *g = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int e = lane + 32 * v;
            if (!RAGGED || e < d4)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                 ring_s + (uint32_t)((slot * SLOT + 32 * v) * 16)),
                             "l"(g + e)
                             : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll
    for (int q = 0; q < NS - 1; ++q)
        issue(reinterpret_cast<const float *>(
                  __shfl_sync(0xffffffffu, (unsigned long long)reinterpret_cast<uintptr_t>(sp), q)),
              q);
    int slot = 0;  // ring slot of the candidate being computed
    uint32_t cur_row = 0xffffffffu;
    float4 a[V];
#pragma unroll
    for (int v = 0; v < V; ++v) a[v] = make_float4(0.f, 0.f, 0.f, 0.f);

    for (;;) {
        const bool has_next = un < units;
        uint64_t unn = units;  // the ticket after the next unit (taken only while units remain)
        // the next unit's lookups (stages 0, R2, R3, FIN); with no next unit they resolve candidate 0
        uint2 nc = make_uint2(0u, 0u);
        bool nok = false;
        uint32_t njob = 0;
        float nia = 0.f, nib = 0.f, nej = 0.f;
        long long nld = 0;
        const float *nS = nullptr;
        uint32_t nx = 0, ngi = 0, ngj = 0;
        const float *nsp = nullptr;
        float nsc = 0.f;
        bool my_emit = false;
        BatchPair my{};
#pragma unroll 1
        for (int j = 0; j < STEPS; ++j) {
            if (j == 0) {
                const uint64_t k = un * 32 + lane;
                nok = has_next && k < n;
                nc = sorted[nok ? k : (has_next ? un * 32 : 0ull)];
            } else if (j == R2) {
                njob = (uint32_t)__ldg(row_job + nc.x);
                nia = invA[nc.x];
                nib = invB[nc.y];
                if (has_next) unn = ticket();
            } else if (j == R3) {
                ngi = batch_row_a(br, nc.x, njob);
                ngj = batch_row_b(br, nc.y, njob);
                nS = br.S[njob];
                nld = br.ldS[njob];
                nej = __ldg(br.eps + njob);
            } else if (j == FIN) {
                nx = nc.x;
                nsp = nS + (int64_t)ngj * nld;
                nsc = nia * nib;
            }
            float part[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const int q = j * C + c;
                // copy the S row of candidate q + NS - 1 into the slot freed by candidate q - 1
                const int qi = q + NS - 1;
                const uintptr_t rp = qi < 32 ? reinterpret_cast<uintptr_t>(sp) : reinterpret_cast<uintptr_t>(nsp);
                issue(reinterpret_cast<const float *>(__shfl_sync(0xffffffffu, (unsigned long long)rp, qi & 31)),
                      slot == 0 ? NS - 1 : slot - 1);
                asm volatile("cp.async.wait_group %0;" ::"n"(NS - 1) : "memory");
                __syncwarp();
                const uint32_t xq = __shfl_sync(0xffffffffu, x, q);
                if (xq != cur_row) {  // warp-uniform: the next A row's run starts
                    cur_row = xq;
                    const uint32_t jq = __shfl_sync(0xffffffffu, job, q);
                    const uint32_t iq = __shfl_sync(0xffffffffu, gi, q);
                    const float4 *ra = reinterpret_cast<const float4 *>(br.R[jq] + (int64_t)iq * br.ldR[jq]);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int e = lane + 32 * v;
                        a[v] = (!RAGGED || e < d4) ? __ldg(ra + e) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                const float4 *b = ring + slot * SLOT + lane;
                float acc = 0.f;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float4 bv = b[32 * v];
                    acc = fmaf(a[v].x, bv.x, acc);
                    acc = fmaf(a[v].y, bv.y, acc);
                    acc = fmaf(a[v].z, bv.z, acc);
                    acc = fmaf(a[v].w, bv.w, acc);
                }
                part[c] = acc;
                __syncwarp();  // every lane is done with the slot before it is refilled
                slot = slot + 1 == NS ? 0 : slot + 1;
            }
            const float tot = transpose_sum<C>(part, lane);
            const int q0 = j * C;
            const float dotv = __shfl_sync(0xffffffffu, tot, ((lane - q0) & (C - 1)) * (32 / C));
            const bool decide = lane >= q0 && lane < q0 + C && ok;
            float sim = fminf(1.f, fmaxf(-1.f, dotv * sc));
            const bool near = decide && fabsf(sim - ej) < fp64_band;
            bool emit = sim >= ej;
            unsigned nm = __ballot_sync(0xffffffffu, near);
            while (nm) {
                const int q = __ffs(nm) - 1;
                nm &= nm - 1u;
                const uint32_t qj = __shfl_sync(0xffffffffu, job, q);
                const uint32_t qi2 = __shfl_sync(0xffffffffu, gi, q);
                const float *qs = reinterpret_cast<const float *>(
                    __shfl_sync(0xffffffffu, (unsigned long long)reinterpret_cast<uintptr_t>(sp), q));
                const double s64 = accurate_cosine(br.R[qj] + (int64_t)qi2 * br.ldR[qj], qs, d, lane);
                if (lane == q) {
                    emit = s64 >= (double)ej;
                    sim = (float)s64;
                }
            }
            if (near) atomicAdd(band_count, 1ull);
            if (decide) {
                my_emit = emit;
                my = BatchPair{job, gi, gj, sim};
            }
        }
        warp_emit_rec<false>(my_emit, my, stg, stg_n, out_count, out, out_cap, 0, lane, false);
        if (!has_next) break;
        u = un;
        un = unn;
        x = nx;
        job = njob;
        gi = ngi;
        gj = ngj;
        sp = nsp;
        sc = nsc;
        ej = nej;
        ok = nok;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    warp_emit_rec<false>(false, BatchPair{}, stg, stg_n, out_count, out, out_cap, 0, lane, true);
}

size_t rescore_stream_batch_buf_bytes(int64_t n_buckets, int64_t rows_a)
{
    const int64_t nb = std::max<int64_t>(1, n_buckets);
    const int64_t scan_blocks = (nb + SCAN_ITEMS - 1) / SCAN_ITEMS;
    return (size_t)(4 * nb + 2 + 2 * scan_blocks + 2 + 2) * sizeof(unsigned long long) +
           (size_t)std::max<int64_t>(1, rows_a) * sizeof(int);
}

template <int V, int C, int NS, bool RAGGED, int CTAS>
static cudaError_t launch_stream_kernel_r(int num_sms, cudaStream_t st, const uint2 *sorted,
                                        const unsigned long long *cand_count, uint64_t cand_cap, const int *row_job,
                                        const BatchRows &br, int d, const float *invA, const float *invB,
                                        float fp64_band, BatchPair *out, uint64_t out_cap,
                                        unsigned long long *out_count, unsigned long long *band_count,
                                        unsigned long long *unit_ticket)
{
    constexpr int MAX_SMEM = 98304;  // eight warps' rings at the widest rows of the instantiation
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!((configured >> dev) & 1ull)) {
        e = cudaFuncSetAttribute(rescore_stream_batch_kernel<V, C, NS, RAGGED, CTAS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_SMEM);
        if (e != cudaSuccess) return e;
        configured |= 1ull << dev;
    }
    const size_t smem = (size_t)RS_WARPS * NS * 32 * V * 16;
    if (smem > (size_t)MAX_SMEM) return cudaErrorInvalidValue;
    const uint64_t units = (cand_cap + 31) / 32;
    const uint64_t blocks = (units + RS_WARPS - 1) / RS_WARPS;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)num_sms * CTAS));
    rescore_stream_batch_kernel<V, C, NS, RAGGED, CTAS><<<grid, RS_WARPS * 32, smem, st>>>(
        sorted, cand_count, cand_cap, row_job, br, d, invA, invB, fp64_band, out, out_cap, out_count, band_count,
        unit_ticket);
    return cudaGetLastError();
}

template <int V, int C, int NS, int CTAS = 2>
static cudaError_t launch_stream_kernel(int num_sms, cudaStream_t st, const uint2 *sorted,
                                        const unsigned long long *cand_count, uint64_t cand_cap, const int *row_job,
                                        const BatchRows &br, int d, const float *invA, const float *invB,
                                        float fp64_band, BatchPair *out, uint64_t out_cap,
                                        unsigned long long *out_count, unsigned long long *band_count,
                                        unsigned long long *unit_ticket)
{
    // rows of exactly 32 V float4 need no zero fill
    if (d == 128 * V)
        return launch_stream_kernel_r<V, C, NS, false, CTAS>(num_sms, st, sorted, cand_count, cand_cap, row_job, br,
                                                             d, invA, invB, fp64_band, out, out_cap, out_count,
                                                             band_count, unit_ticket);
    return launch_stream_kernel_r<V, C, NS, true, CTAS>(num_sms, st, sorted, cand_count, cand_cap, row_job, br, d, invA,
                                                        invB, fp64_band, out, out_cap, out_count, band_count,
                                                        unit_ticket);
}

cudaError_t launch_rescore_stream_batch(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                        uint2 *sorted, void *buf, int64_t rows_a, const BatchRows &br,
                                        const long long *bbase, const int *nA, int64_t n_buckets, int64_t sblock_rows,
                                        int d, const float *invA, const float *invB, float fp64_band, BatchPair *out,
                                        uint64_t out_cap, unsigned long long *out_count,
                                        unsigned long long *band_count, int num_sms, cudaStream_t st)
{
    if (cand_cap == 0) return cudaSuccess;
    if (d % 4 != 0 || d > 1024 || !sorted || !buf || rows_a < 1 || n_buckets < 1 || n_buckets >= 0xffffffffll ||
        sblock_rows < 1 || sblock_rows > 0x7fffffffll)
        return cudaErrorInvalidValue;
    const int64_t nb = n_buckets;
    const int64_t scan_blocks = (nb + SCAN_ITEMS - 1) / SCAN_ITEMS;
    unsigned long long *cnt = static_cast<unsigned long long *>(buf);
    unsigned long long *off = cnt + nb;        // nb + 1
    unsigned long long *cursor = off + nb + 1;  // nb
    unsigned long long *choff = cursor + nb;    // nb + 1
    unsigned long long *tot = choff + nb + 1;    // 2 * scan_blocks + 2
    unsigned long long *unit_ticket = tot + 2 * scan_blocks + 2;           // 2 (one used)
    int *row_job = reinterpret_cast<int *>(unit_ticket + 2);              // rows_a
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)nb * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(unit_ticket, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    panel_job_kernel<<<(unsigned)((rows_a + 255) / 256), 256, 0, st>>>(br.a_off, br.n_jobs, 0, rows_a, row_job);
    const JobBlockBucket bucket{row_job, bbase, br.a_off, br.b_off, nA, (unsigned)sblock_rows};
    const unsigned gs = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((cand_cap + 255) / 256, (uint64_t)num_sms * 8));
    panel_hist_kernel<<<gs, 256, 0, st>>>(cand, cand_count, cand_cap, bucket, cnt);
    panel_scan_reduce_kernel<<<(unsigned)scan_blocks, SCAN_THREADS, 0, st>>>(cnt, nb, tot);
    panel_scan_top_kernel<<<1, SCAN_THREADS, 0, st>>>(tot, (int)scan_blocks);
    panel_scan_down_kernel<<<(unsigned)scan_blocks, SCAN_THREADS, 0, st>>>(cnt, nb, tot, off, cursor, choff);
    panel_scatter_kernel<<<gs, 256, 0, st>>>(cand, cand_count, cand_cap, bucket, cursor, sorted);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
#define EJ_SB_ARGS \
    num_sms, st, sorted, cand_count, cand_cap, row_job, br, d, invA, invB, fp64_band, out, out_cap, out_count, band_count, \
        unit_ticket
    if (d <= 128) return launch_stream_kernel<1, 8, 8>(EJ_SB_ARGS);
    if (d <= 256) return launch_stream_kernel<2, 4, 8>(EJ_SB_ARGS);
    if (d <= 384) return launch_stream_kernel<3, 4, 8>(EJ_SB_ARGS);
    if (d <= 512) return launch_stream_kernel<4, 2, 6>(EJ_SB_ARGS);
    if (d <= 768) return launch_stream_kernel<6, 2, 4>(EJ_SB_ARGS);
    return launch_stream_kernel<8, 1, 3>(EJ_SB_ARGS);
#undef EJ_SB_ARGS
}

}  // namespace ej
