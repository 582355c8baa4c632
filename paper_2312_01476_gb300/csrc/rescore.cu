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
            gi = (uint32_t)(c.x - __ldg(br.a_off + lo));
            gj = (uint32_t)(c.y - __ldg(br.b_off + lo));
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

cudaError_t launch_rescore(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap, const float *R,
                           int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *idsR,
                           const uint32_t *idsS, const float *invR, const float *invS, float eps, float fp64_band,
                           ejoin_pair *out, uint64_t out_cap, unsigned long long *out_count,
                           unsigned long long *band_count, int count_only, int num_sms, cudaStream_t st,
                           uint2 *band_list, uint64_t band_cap, int mirror)
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
    if (e != cudaSuccess || fp64_band <= 0.f) return e;
    // the accurate tier over the candidates listed near eps (stream order: after the FP32 tier)
    const unsigned gb = (unsigned)std::min<uint64_t>((band_cap + 255) / 256, (uint64_t)num_sms * 8);
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
#undef EJ_RESCORE_ARGS
    return cudaGetLastError();
}

}  // namespace ej
