// FP32 CUDA-core similarity contraction with fused threshold and compaction
// (the plain FP32 path, and the GPU correctness reference for the tensor-core
// kernels).
//
// Tensor formulation of Sec. IV-C: D = R S^T over normalised rows, formed
// block by block (Eq. Block Matrix Dot Product Decomposition) in 128 x 128
// tiles whose K loop runs over 16-wide slices of the padded dimension.  D is
// never written (Sec. V-B, memory-bounded evaluation): each tile is compared
// against the candidate threshold in registers (Sec. III-B threshold
// predicate) and the positions of the passing entries are appended to the
// candidate buffer (Sec. IV-C, mapping back through partition offsets).  One
// global atomic per tile claims space for all of the tile's candidates.
#include "ejoin_internal.cuh"

namespace ej {

namespace {
constexpr int BM = 128, BN = 128, BK = 16, NT = 256, PAD = 4;
}

__global__ void __launch_bounds__(NT, 2) sim_simt_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                         int kp, const long long *__restrict__ nA_ptr,
                                                         const long long *__restrict__ nB_ptr, float thr,
                                                         uint2 *__restrict__ cand, uint64_t cap,
                                                         unsigned long long *cand_count, int count_only)
{
    __shared__ __align__(16) float As[BK][BM + PAD];
    __shared__ __align__(16) float Bs[BK][BN + PAD];
    __shared__ int warp_cnt[NT / 32];
    __shared__ unsigned long long tile_base;

    const int64_t nA = *nA_ptr, nB = *nB_ptr;
    const int64_t tiles_m = (nA + BM - 1) / BM, tiles_n = (nB + BN - 1) / BN;
    const int64_t total = tiles_m * tiles_n;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int lane = tid & 31, warp = tid >> 5;

    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int64_t m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

        // global -> register staging: 2 float4 of A and 2 of B per thread per slice
        float4 ra[2], rb[2];
        auto gload = [&](int k0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int idx = tid + h * NT;  // 0..511
                const int row = idx >> 2, kq = idx & 3;
                ra[h] = *reinterpret_cast<const float4 *>(A + (m0 + row) * (int64_t)kp + k0 + 4 * kq);
                rb[h] = *reinterpret_cast<const float4 *>(B + (n0 + row) * (int64_t)kp + k0 + 4 * kq);
            }
        };
        auto sstore = [&]() {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int idx = tid + h * NT;
                const int row = idx >> 2, kq = idx & 3;
                As[4 * kq + 0][row] = ra[h].x;
                As[4 * kq + 1][row] = ra[h].y;
                As[4 * kq + 2][row] = ra[h].z;
                As[4 * kq + 3][row] = ra[h].w;
                Bs[4 * kq + 0][row] = rb[h].x;
                Bs[4 * kq + 1][row] = rb[h].y;
                Bs[4 * kq + 2][row] = rb[h].z;
                Bs[4 * kq + 3][row] = rb[h].w;
            }
        };

        gload(0);
        for (int k0 = 0; k0 < kp; k0 += BK) {
            __syncthreads();
            sstore();
            __syncthreads();
            if (k0 + BK < kp) gload(k0 + BK);
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
        }

        // ---- epilogue: threshold compare, then one atomic per tile
        unsigned long long mask = 0ull;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int64_t col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
                if (row < nA && col < nB && acc[i][j] >= thr) mask |= 1ull << (i * 8 + j);
            }
        }
        const int cnt = __popcll(mask);
        if (__syncthreads_or(cnt)) {
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) warp_cnt[warp] = incl;
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int w = 0; w < NT / 32; ++w) {
                    const int c = warp_cnt[w];
                    warp_cnt[w] = run;
                    run += c;
                }
                tile_base = atomicAdd(cand_count, (unsigned long long)run);
            }
            __syncthreads();
            if (!count_only) {
                unsigned long long pos = tile_base + warp_cnt[warp] + (incl - cnt);
                while (mask) {
                    const int b = __ffsll(mask) - 1;
                    mask &= mask - 1;
                    const int i = b >> 3, j = b & 7;
                    const int64_t row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
                    const int64_t col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
                    if (pos < cap) cand[pos] = make_uint2((uint32_t)row, (uint32_t)col);
                    ++pos;
                }
            }
        }
    }
}

cudaError_t launch_sim_simt(const float *A, const float *B, int kp, const long long *nA, const long long *nB,
                            float thr, uint2 *cand, uint64_t cap, unsigned long long *cand_count, int count_only,
                            int num_sms, cudaStream_t st)
{
    sim_simt_kernel<<<num_sms * 2, NT, 0, st>>>(A, B, kp, nA, nB, thr, cand, cap, cand_count, count_only);
    return cudaGetLastError();
}

}  // namespace ej
