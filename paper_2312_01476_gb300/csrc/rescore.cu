// Exact re-score of the contraction's candidates (guard band around eps).
//
// Every candidate (a pair whose bulk-precision similarity reached eps - band)
// gets its similarity recomputed from the original FP32 rows (Sec. III-A,
// Eq. (Cosine Similarity)): an FP32 dot product, lane-parallel with a
// butterfly reduction, scaled by the two FP32 inverse norms from the
// normalisation pass.  A candidate whose FP32 similarity lies within
// fp64_band of eps is recomputed again in FP64 (dot product and both norms).
// Pairs with sim >= eps (Sec. III-B threshold predicate) are emitted as
// (original i, original j, sim) records (Sec. IV-C, mapping back to tuples),
// one global atomic per block of candidates.
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

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(RS_WARPS * 32) rescore_kernel(
    const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_count, uint64_t cand_cap,
    const float *__restrict__ R, int64_t ldR, const float *__restrict__ S, int64_t ldS, int d,
    const uint32_t *__restrict__ idsR, const uint32_t *__restrict__ idsS, const float *__restrict__ invR,
    const float *__restrict__ invS, float eps, float fp64_band, ejoin_pair *__restrict__ out, uint64_t out_cap,
    unsigned long long *out_count, unsigned long long *band_count, int count_only)
{
    __shared__ int wcnt[RS_WARPS];
    __shared__ unsigned long long base_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t n = *cand_count;
    if (n > cand_cap) n = cand_cap;
    const bool vec = ((ldR & 3) == 0) && ((ldS & 3) == 0) && ((reinterpret_cast<uintptr_t>(R) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(S) & 15) == 0);
    const int d4 = vec ? (d >> 2) : 0;  // float4 groups
    const double eps_d = (double)eps;

    for (uint64_t blk = (uint64_t)blockIdx.x * RS_PER_BLOCK; blk < n; blk += (uint64_t)gridDim.x * RS_PER_BLOCK) {
        // lane q (< RS_PER_WARP) holds the outcome of the warp's q-th candidate
        bool my_emit = false;
        uint32_t my_i = 0, my_j = 0;
        float my_sim = 0.f;
        int my_band = 0;
        const uint64_t wbase = blk + (uint64_t)warp * RS_PER_WARP;
        for (int q = 0; q < RS_PER_WARP; ++q) {
            const uint64_t k = wbase + q;
            if (k >= n) break;  // warp-uniform
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
            int band = 0;
            if (fabsf(sim - eps) < fp64_band) {
                // FP64 tier: dot product and both norms in double
                double dd = 0.0, nr = 0.0, ns = 0.0;
                for (int kk = lane; kk < d; kk += 32) {
                    const double a = (double)__ldg(r + kk), b = (double)__ldg(s + kk);
                    dd = fma(a, b, dd);
                    nr = fma(a, a, nr);
                    ns = fma(b, b, ns);
                }
                dd = warp_sum_d(dd);
                nr = warp_sum_d(nr);
                ns = warp_sum_d(ns);
                double s64 = (nr > 0.0 && ns > 0.0) ? dd / (sqrt(nr) * sqrt(ns)) : 0.0;
                s64 = fmin(1.0, fmax(-1.0, s64));
                emit = s64 >= eps_d;
                sim = (float)s64;
                band = 1;
            }
            if (lane == q) {
                my_emit = emit;
                my_i = i;
                my_j = j;
                my_sim = sim;
                my_band = band;
            }
        }
        // block-level aggregation of the emitted pairs: one atomic per block step
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
        if (my_emit && !count_only) {
            const unsigned long long pos = base_s + wcnt[warp] + __popc(m & ((1u << lane) - 1u));
            if (pos < out_cap) {
                ejoin_pair p;
                p.i = my_i;
                p.j = my_j;
                p.sim = my_sim;
                out[pos] = p;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_rescore(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap, const float *R,
                           int64_t ldR, const float *S, int64_t ldS, int d, const uint32_t *idsR,
                           const uint32_t *idsS, const float *invR, const float *invS, float eps, float fp64_band,
                           ejoin_pair *out, uint64_t out_cap, unsigned long long *out_count,
                           unsigned long long *band_count, int count_only, int num_sms, cudaStream_t st)
{
    if (cand_cap == 0) return cudaSuccess;
    uint64_t blocks = (cand_cap + RS_PER_BLOCK - 1) / RS_PER_BLOCK;
    const uint64_t lim = (uint64_t)num_sms * 8;
    if (blocks > lim) blocks = lim;
    rescore_kernel<<<(unsigned)blocks, RS_WARPS * 32, 0, st>>>(cand, cand_count, cand_cap, R, ldR, S, ldS, d, idsR,
                                                               idsS, invR, invS, eps, fp64_band, out, out_cap,
                                                               out_count, band_count, count_only);
    return cudaGetLastError();
}

}  // namespace ej
