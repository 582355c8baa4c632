// Kernels of the learned sketch network (768 -> 256 -> 64, GELU, unit-length
// output) used by the learned tile pruning: forward, pair loss, backward and
// Adam, all FP32 on CUDA cores.  The paper has no learned component; this is
// the "learned pruning" form of the join.
//
//   a = W1 x + b1,  h = GELU(a) = a Phi(a),  z = W2 h + b2,  s = z / |z|
//   loss = sum_k w_k (s_pk . s_qk - t_k)^2 / sum_k w_k
//
// The contractions are small next to the join (about 0.43 MFLOP per row), so
// one generic tiled GEMM with gathered / scaled rows, a fused bias + GELU
// epilogue and a split-K mode covers every product of the forward and
// backward passes.
#include "mlp_internal.cuh"

namespace ej {

namespace {
constexpr int GT = 64;   // output tile (GT x GT)
constexpr int GK = 16;   // K slice
constexpr int GNT = 256; // threads: 16 x 16, 4 x 4 outputs each

__device__ __forceinline__ float gelu_f(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float a)
{
    return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}
}  // namespace

__global__ void __launch_bounds__(GNT) gemm_f32_kernel(const GemmArgs g)
{
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * GT, n0 = (int64_t)blockIdx.x * GT;
    const int64_t k_begin = (int64_t)blockIdx.z * g.k_chunk;
    int64_t k_end = k_begin + g.k_chunk;
    if (k_end > g.K) k_end = g.K;
    const bool a_kfast = g.a_cs == 1;  // A(i, k) contiguous along k
    const bool b_nfast = g.b_cs == 1;  // B(k, j) contiguous along j
    float acc[4][4] = {};

    for (int64_t k0 = k_begin; k0 < k_end; k0 += GK) {
#pragma unroll
        for (int r = 0; r < (GT * GK) / GNT; ++r) {
            const int e = tid + r * GNT;
            const int row = a_kfast ? (e / GK) : (e % GT);
            const int kk = a_kfast ? (e % GK) : (e / GT);
            const int64_t gi = m0 + row, gk = k0 + kk;
            float v = 0.f;
            if (gi < g.M && gk < k_end) {
                const int64_t ar = g.aidx ? (int64_t)g.aidx[gi] : gi;
                v = g.A[ar * g.a_rs + gk * g.a_cs];
                if (g.ascale) v *= g.ascale[ar];
            }
            As[kk][row] = v;
        }
#pragma unroll
        for (int r = 0; r < (GT * GK) / GNT; ++r) {
            const int e = tid + r * GNT;
            const int col = b_nfast ? (e % GT) : (e / GK);
            const int kk = b_nfast ? (e / GT) : (e % GK);
            const int64_t gj = n0 + col, gk = k0 + kk;
            float v = 0.f;
            if (gj < g.N && gk < k_end) {
                const int64_t br = g.bidx ? (int64_t)g.bidx[gk] : gk;
                v = g.B[br * g.b_rs + gj * g.b_cs];
                if (g.bscale) v *= g.bscale[br];
            }
            Bs[kk][col] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = m0 + ty * 4 + i;
        if (row >= g.M) continue;
        const float rs = g.rowscale ? g.rowscale[g.aidx ? g.aidx[row] : row] : 1.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t col = n0 + tx * 4 + j;
            if (col >= g.N) continue;
            float v = acc[i][j] * rs;
            float *cp = g.C + row * g.ldc + col;
            if (g.atomic_acc) {
                atomicAdd(cp, v);
                continue;
            }
            if (g.bias) v += g.bias[col];
            if (g.pre) g.pre[row * g.ldc + col] = v;
            if (g.act == ACT_GELU) v = gelu_f(v);
            *cp = v;
        }
    }
}

// Inference form of the layer product: C[i][j] = act(rowscale[i] * sum_k A[i][k] W[j][k] + bias[j]) with A
// (M x K) and W (N x K) both contiguous along k, K % 16 == 0, lda, ldw % 4 == 0 and 16-byte aligned rows.
// 128 x 128 output tile per block, 8 x 8 outputs per thread (two LDS.128 of A and two of W per k feed 64
// FMAs), float4 global loads along k into k-major shared memory, and the next 16-wide K slice prefetched
// into registers during the current one.
constexpr int NT_T = 128, NT_K = 16;

__global__ void __launch_bounds__(256) gemm_nt_f32_kernel(const float *__restrict__ A, int64_t lda,
                                                          const float *__restrict__ W, int64_t ldw,
                                                          const float *__restrict__ bias,
                                                          const float *__restrict__ rowscale, int act,
                                                          float *__restrict__ C, int64_t ldc, int64_t M, int N,
                                                          int K)
{
    __shared__ __align__(16) float As[NT_K][NT_T + 4];
    __shared__ __align__(16) float Ws[NT_K][NT_T + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * NT_T;
    const int n0 = blockIdx.x * NT_T;
    // loader: thread -> rows lr and lr + 64 of the tile, k quad lq (4 floats) of the slice
    const int lr = tid >> 2, lq = (tid & 3) * 4;
    auto load = [&](int k0, float4 (&a)[2], float4 (&w)[2]) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gi = m0 + lr + 64 * h;
            const int gj = n0 + lr + 64 * h;
            a[h] = gi < M ? __ldg(reinterpret_cast<const float4 *>(A + gi * lda + k0 + lq))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
            w[h] = gj < N ? __ldg(reinterpret_cast<const float4 *>(W + (int64_t)gj * ldw + k0 + lq))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    float acc[8][8] = {};
    float4 ra[2], rw[2];
    load(0, ra, rw);
    for (int k0 = 0; k0 < K; k0 += NT_K) {
        __syncthreads();  // the previous slice has been consumed
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = lr + 64 * h;
            As[lq + 0][r] = ra[h].x;
            As[lq + 1][r] = ra[h].y;
            As[lq + 2][r] = ra[h].z;
            As[lq + 3][r] = ra[h].w;
            Ws[lq + 0][r] = rw[h].x;
            Ws[lq + 1][r] = rw[h].y;
            Ws[lq + 2][r] = rw[h].z;
            Ws[lq + 3][r] = rw[h].w;
        }
        __syncthreads();
        if (k0 + NT_K < K) load(k0 + NT_K, ra, rw);
#pragma unroll
        for (int kk = 0; kk < NT_K; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
            const float4 w0 = *reinterpret_cast<const float4 *>(&Ws[kk][tx * 4]);
            const float4 w1 = *reinterpret_cast<const float4 *>(&Ws[kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], wv[j], acc[i][j]);
        }
    }
    // outputs: rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns tx*4 + {0..3} and 64 + tx*4 + {0..3}
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t row = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= M) continue;
        const float rs = rowscale ? rowscale[row] : 1.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (col >= N) continue;
            float v = acc[i][j] * rs;
            if (bias) v += bias[col];
            if (act == ACT_GELU) v = gelu_f(v);
            C[row * ldc + col] = v;
        }
    }
}

cudaError_t launch_gemm_nt_f32(const float *A, int64_t lda, const float *W, int64_t ldw, const float *bias,
                               const float *rowscale, int act, float *C, int64_t ldc, int64_t M, int N, int K,
                               cudaStream_t st)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K % NT_K || lda % 4 || ldw % 4 || (reinterpret_cast<uintptr_t>(A) & 15) ||
        (reinterpret_cast<uintptr_t>(W) & 15))
        return cudaErrorInvalidValue;
    const int64_t max_rows = (int64_t)65535 * NT_T;
    for (int64_t r0 = 0; r0 < M; r0 += max_rows) {
        const int64_t m = std::min<int64_t>(max_rows, M - r0);
        dim3 grid((unsigned)((N + NT_T - 1) / NT_T), (unsigned)((m + NT_T - 1) / NT_T));
        gemm_nt_f32_kernel<<<grid, 256, 0, st>>>(A + r0 * lda, lda, W, ldw, bias, rowscale ? rowscale + r0 : nullptr,
                                                 act, C + r0 * ldc, ldc, m, N, K);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gemm_f32(const GemmArgs &g, int num_sms, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    GemmArgs a = g;
    const int64_t tiles = ((g.M + GT - 1) / GT) * ((g.N + GT - 1) / GT);
    int64_t splits = 1;
    if (g.atomic_acc) {
        // spread a long K over enough CTAs to fill the GPU (output pre-zeroed by the caller)
        splits = std::max<int64_t>(1, std::min<int64_t>((4 * num_sms + tiles - 1) / tiles, (g.K + 255) / 256));
    }
    a.k_chunk = ((g.K + splits - 1) / splits + GK - 1) / GK * GK;
    if (a.k_chunk <= 0) a.k_chunk = GK;
    splits = (g.K + a.k_chunk - 1) / a.k_chunk;
    if (splits < 1) splits = 1;
    // the grid's y dimension is limited to 65,535 blocks: larger M runs in row chunks
    const int64_t max_rows = (int64_t)65535 * GT;
    for (int64_t r0 = 0; r0 < g.M; r0 += max_rows) {
        GemmArgs c = a;
        c.M = std::min<int64_t>(max_rows, g.M - r0);
        if (g.aidx) {
            c.aidx = g.aidx + r0;
        } else {
            c.A = g.A + r0 * g.a_rs;
            if (g.rowscale) c.rowscale = g.rowscale + r0;
            if (g.ascale) c.ascale = g.ascale + r0;
        }
        c.C = g.C + r0 * g.ldc;
        if (g.pre) c.pre = g.pre + r0 * g.ldc;
        dim3 grid((unsigned)((g.N + GT - 1) / GT), (unsigned)((c.M + GT - 1) / GT), (unsigned)splits);
        gemm_f32_kernel<<<grid, GNT, 0, st>>>(c);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// s = z / |z| per row (one warp per row); keeps |z| for the backward pass.
__global__ void rownorm_kernel(const float *__restrict__ z, int64_t n, int k, float *__restrict__ s,
                               float *__restrict__ nz)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        float ss = 0.f;
        for (int c = lane; c < k; c += 32) ss = fmaf(z[r * k + c], z[r * k + c], ss);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float nrm = sqrtf(ss);
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        for (int c = lane; c < k; c += 32) s[r * k + c] = z[r * k + c] * inv;
        if (lane == 0 && nz) nz[r] = nrm;
    }
}

// Pair k = rows (k, B + k): c = s_p . s_q, g = 2 w (c - t) / wsum, ds_p = g s_q, ds_q = g s_p.
__global__ void pair_grad_kernel(const float *__restrict__ s, int64_t B, int k, const float *__restrict__ t,
                                 const float *__restrict__ w, const float *__restrict__ wsum, float *__restrict__ ds,
                                 float *__restrict__ loss)
{
    const float inv_wsum = *wsum > 0.f ? 1.f / *wsum : 0.f;
    const int lane = threadIdx.x & 31;
    const int64_t wp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float lsum = 0.f;
    for (int64_t p = wp; p < B; p += nw) {
        const float *sp = s + p * k, *sq = s + (B + p) * k;
        float c = 0.f;
        for (int j = lane; j < k; j += 32) c = fmaf(sp[j], sq[j], c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        const float e = c - t[p];
        const float gk = 2.f * w[p] * e * inv_wsum;
        if (ds) {
            for (int j = lane; j < k; j += 32) {
                ds[p * k + j] = gk * sq[j];
                ds[(B + p) * k + j] = gk * sp[j];
            }
        }
        lsum += w[p] * e * e * inv_wsum;
    }
    if (lane == 0 && loss) atomicAdd(loss, lsum);
}

// out[k] = s_p . s_q for pair k = rows (k, B + k).
__global__ void pair_dot_kernel(const float *__restrict__ s, int64_t B, int k, float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t wp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = wp; p < B; p += nw) {
        float c = 0.f;
        for (int j = lane; j < k; j += 32) c = fmaf(s[p * k + j], s[(B + p) * k + j], c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) out[p] = c;
    }
}

// 1 / |x| per row (one warp per row, FP32; 0 for a zero row).
__global__ void row_inv_norm_kernel(const float *__restrict__ x, int64_t n, int d, int64_t ld, float *__restrict__ inv)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        float ss = 0.f;
        for (int c = lane; c < d; c += 32) ss = fmaf(x[r * ld + c], x[r * ld + c], ss);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) inv[r] = ss > 0.f ? 1.f / sqrtf(ss) : 0.f;
    }
}

// dz = (ds - s (s . ds)) / |z| per row.
__global__ void rownorm_backward_kernel(const float *__restrict__ s, const float *__restrict__ ds,
                                        const float *__restrict__ nz, int64_t n, int k, float *__restrict__ dz)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        float dot = 0.f;
        for (int c = lane; c < k; c += 32) dot = fmaf(s[r * k + c], ds[r * k + c], dot);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const float inv = nz[r] > 0.f ? 1.f / nz[r] : 0.f;
        for (int c = lane; c < k; c += 32) dz[r * k + c] = (ds[r * k + c] - s[r * k + c] * dot) * inv;
    }
}

// dh <- dh * GELU'(a), elementwise.
__global__ void gelu_backward_kernel(float *__restrict__ dh, const float *__restrict__ a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dh[i] *= gelu_grad_f(a[i]);
}

// out[c] += sum_r x[r * k + c] over a chunk of rows (out pre-zeroed).
__global__ void colsum_kernel(const float *__restrict__ x, int64_t n, int k, int64_t rows_per_block,
                              float *__restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
    int64_t r1 = r0 + rows_per_block;
    if (r1 > n) r1 = n;
    float acc = 0.f;
    for (int64_t r = r0; r < r1; ++r) acc += x[r * k + c];
    atomicAdd(out + c, acc);
}

// Adam step: m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2; p -= lr mhat / (sqrt(vhat) + eps).
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static unsigned blocks_for(int64_t work, int per_block, int num_sms)
{
    int64_t b = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

cudaError_t launch_rownorm(const float *z, int64_t n, int k, float *s, float *nz, int num_sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    rownorm_kernel<<<blocks_for(n, 8, num_sms), 256, 0, st>>>(z, n, k, s, nz);
    return cudaGetLastError();
}

cudaError_t launch_pair_grad(const float *s, int64_t B, int k, const float *t, const float *w, const float *wsum,
                             float *ds, float *loss, int num_sms, cudaStream_t st)
{
    if (B <= 0) return cudaSuccess;
    pair_grad_kernel<<<blocks_for(B, 8, num_sms), 256, 0, st>>>(s, B, k, t, w, wsum, ds, loss);
    return cudaGetLastError();
}

cudaError_t launch_pair_dot(const float *s, int64_t B, int k, float *out, int num_sms, cudaStream_t st)
{
    if (B <= 0) return cudaSuccess;
    pair_dot_kernel<<<blocks_for(B, 8, num_sms), 256, 0, st>>>(s, B, k, out);
    return cudaGetLastError();
}

cudaError_t launch_row_inv_norm(const float *x, int64_t n, int d, int64_t ld, float *inv, int num_sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    row_inv_norm_kernel<<<blocks_for(n, 8, num_sms), 256, 0, st>>>(x, n, d, ld, inv);
    return cudaGetLastError();
}

cudaError_t launch_rownorm_backward(const float *s, const float *ds, const float *nz, int64_t n, int k, float *dz,
                                    int num_sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    rownorm_backward_kernel<<<blocks_for(n, 8, num_sms), 256, 0, st>>>(s, ds, nz, n, k, dz);
    return cudaGetLastError();
}

cudaError_t launch_gelu_backward(float *dh, const float *a, int64_t n, int num_sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    gelu_backward_kernel<<<blocks_for(n, 256, num_sms), 256, 0, st>>>(dh, a, n);
    return cudaGetLastError();
}

cudaError_t launch_colsum(const float *x, int64_t n, int k, float *out, int num_sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t chunks = std::max<int64_t>(1, std::min<int64_t>(4 * num_sms, (n + 255) / 256));
    const int64_t rpb = (n + chunks - 1) / chunks;
    dim3 grid((unsigned)((k + 127) / 128), (unsigned)((n + rpb - 1) / rpb));
    colsum_kernel<<<grid, 128, 0, st>>>(x, n, k, rpb, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, int step, int num_sms, cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<blocks_for(n, 256, num_sms), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace ej
