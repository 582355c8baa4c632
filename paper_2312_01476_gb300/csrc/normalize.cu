// Selection pushdown and row normalisation (HBM-bound passes).
//
// Selection (Sec. III-C, Eq. (Selection); pushed below the embedding work as
// in Eq. (E-Selection), and applied as a relational pre-filter in Sec. VI-E):
// an order-preserving stream compaction of the kept row ids in three passes
// (per-block count, one-block scan of the block counts, per-block scatter).
//
// Normalisation (Sec. IV-C: cosine similarity equals the dot product of
// normalised vectors; each row is normalised exactly once, the "prefetch"
// formulation of Sec. IV-A, Eq. nlj-prefetch): one warp per kept row, FP32
// sum of squares accumulated per lane then by a butterfly tree, y = x / ||x||
// (0 for a zero row), stored as FP32 / BF16 / e4m3 with zero padding to the
// contraction's K granularity.
#include "ejoin_internal.cuh"

namespace ej {

__device__ __forceinline__ int block_sum(int v, int *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(SEL_THREADS) sel_count_kernel(SelArgs s, int64_t n, uint32_t *block_counts)
{
    __shared__ int red[SEL_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SEL_ROWS_PER_BLOCK;
    int cnt = 0;
#pragma unroll 4
    for (int it = 0; it < SEL_ITEMS; ++it) {
        const int64_t r = base + (int64_t)it * SEL_THREADS + threadIdx.x;
        if (r < n && sel_keep(s, r)) ++cnt;
    }
    cnt = block_sum(cnt, red);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = (uint32_t)cnt;
}

// Exclusive scan of the per-block counts by one block; writes the total.
__global__ void __launch_bounds__(1024) sel_scan_kernel(const uint32_t *counts, int64_t nb, uint32_t *offsets,
                                                        long long *n_sel)
{
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        unsigned long long v = i < nb ? counts[i] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const unsigned long long warp_excl = warp ? warp_tot[warp - 1] : 0ull;
        if (i < nb) offsets[i] = (uint32_t)(carry + warp_excl + x - v);
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_sel = (long long)carry;
}

__global__ void __launch_bounds__(SEL_THREADS) sel_scatter_kernel(SelArgs s, int64_t n, const uint32_t *offsets,
                                                                  uint32_t *ids)
{
    __shared__ int wcount[SEL_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SEL_ROWS_PER_BLOCK;
    uint32_t running = offsets[blockIdx.x];
    for (int it = 0; it < SEL_ITEMS; ++it) {
        const int64_t r = base + (int64_t)it * SEL_THREADS + threadIdx.x;
        const bool k = r < n && sel_keep(s, r);
        const unsigned m = __ballot_sync(0xffffffffu, k);
        if (lane == 0) wcount[warp] = __popc(m);
        __syncthreads();
        uint32_t before = 0, strip = 0;
        for (int w = 0; w < SEL_THREADS / 32; ++w) {
            const int c = wcount[w];
            before += (w < warp) ? c : 0;
            strip += c;
        }
        if (k) ids[running + before + __popc(m & ((1u << lane) - 1u))] = (uint32_t)r;
        running += strip;
        __syncthreads();
    }
}

__global__ void set_count_kernel(long long *p, long long v) { *p = v; }

// Normalise one row (one warp): y = x / ||x|| (0 for a zero row), written as
// FMT with zero padding to kp; 1/||x|| and the e4m3 scale are written by lane 0.
// raw (optional): the row's d FP32 values are also copied there as read (the
// copy of a row that sits in host memory, for kernels that gather rows later).
template <int FMT>
__device__ __forceinline__ void normalize_row(const float *__restrict__ src, int d, bool vec, void *__restrict__ out,
                                              int64_t c, int64_t ld_out, int kp, float *__restrict__ inv_norm,
                                              float *__restrict__ scale, unsigned *status, int lane,
                                              float *__restrict__ raw = nullptr, bool raw_vec = false)
{
    const int groups = kp >> 2;  // kp is a multiple of 32
    auto load4 = [&](int k) -> float4 {
        float4 v;
        if (vec && k + 3 < d) {
            v = __ldg(reinterpret_cast<const float4 *>(src + k));
        } else {
            v.x = k + 0 < d ? __ldg(src + k + 0) : 0.f;
            v.y = k + 1 < d ? __ldg(src + k + 1) : 0.f;
            v.z = k + 2 < d ? __ldg(src + k + 2) : 0.f;
            v.w = k + 3 < d ? __ldg(src + k + 3) : 0.f;
        }
        return v;
    };

    // pass 1: sum of squares and max |x| (and the raw copy)
    float ss = 0.f, mx = 0.f;
    for (int g = lane; 4 * g < d; g += 32) {
        const float4 v = load4(4 * g);
        if (raw) {
            const int k = 4 * g;
            if (raw_vec && k + 3 < d) {
                *reinterpret_cast<float4 *>(raw + k) = v;
            } else {
                raw[k] = v.x;
                if (k + 1 < d) raw[k + 1] = v.y;
                if (k + 2 < d) raw[k + 2] = v.z;
                if (k + 3 < d) raw[k + 3] = v.w;
            }
        }
        ss = fmaf(v.x, v.x, ss);
        ss = fmaf(v.y, v.y, ss);
        ss = fmaf(v.z, v.z, ss);
        ss = fmaf(v.w, v.w, ss);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    float inv;
    bool bad = false;
    if (isnan(ss) || !isfinite(mx)) {
        // NaN or Inf in the row (fmaxf drops NaN, the sum of squares keeps it)
        bad = true;
        inv = 0.f;
    } else if (isfinite(ss) && (ss >= 0x1p-100f || mx == 0.f)) {
        inv = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
    } else {
        // overflow or underflow of the plain sum: rescale by max |x|
        const float rm = 1.0f / mx;
        float s2 = 0.f;
        for (int g = lane; 4 * g < d; g += 32) {
            const float4 v = load4(4 * g);
            s2 = fmaf(v.x * rm, v.x * rm, s2);
            s2 = fmaf(v.y * rm, v.y * rm, s2);
            s2 = fmaf(v.z * rm, v.z * rm, s2);
            s2 = fmaf(v.w * rm, v.w * rm, s2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        inv = (1.0f / sqrtf(s2)) / mx;
    }
    if (bad && lane == 0) atomicOr(status, ERR_NONFINITE);

    float sc = 1.f, rsc = 1.f;
    if (FMT == FMT_FP8) {
        const float ymax = mx * inv;  // max |y|
        sc = ymax > 0.f ? ymax / 448.f : 1.f;
        rsc = 1.0f / sc;
        if (lane == 0) scale[c] = sc;
    }
    if (lane == 0 && inv_norm) inv_norm[c] = inv;

    // pass 2: write the normalised row, zero padded to kp (out == nullptr: norms and scales only)
    if (!out) return;
    for (int g = lane; g < groups; g += 32) {
        const int k = 4 * g;
        float4 v = k < d ? load4(k) : make_float4(0.f, 0.f, 0.f, 0.f);
        v.x *= inv;
        v.y *= inv;
        v.z *= inv;
        v.w *= inv;
        if (FMT == FMT_F32) {
            float *o = reinterpret_cast<float *>(out) + c * ld_out + k;
            *reinterpret_cast<float4 *>(o) = v;
        } else if (FMT == FMT_BF16) {
            __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(out) + c * ld_out + k;
            __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y);
            __nv_bfloat162 hi = __floats2bfloat162_rn(v.z, v.w);
            uint2 u;
            u.x = *reinterpret_cast<uint32_t *>(&lo);
            u.y = *reinterpret_cast<uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(o) = u;
        } else {
            __nv_fp8_storage_t *o = reinterpret_cast<__nv_fp8_storage_t *>(out) + c * ld_out + k;
            const __nv_fp8x2_storage_t lo =
                __nv_cvt_float2_to_fp8x2(make_float2(v.x * rsc, v.y * rsc), __NV_SATFINITE, __NV_E4M3);
            const __nv_fp8x2_storage_t hi =
                __nv_cvt_float2_to_fp8x2(make_float2(v.z * rsc, v.w * rsc), __NV_SATFINITE, __NV_E4M3);
            *reinterpret_cast<uint32_t *>(o) = (uint32_t)lo | ((uint32_t)hi << 16);
        }
    }
}

// One warp per kept row c: source row ids[c] (or c), output row c.
template <int FMT>
__global__ void __launch_bounds__(256) normalize_kernel(const float *__restrict__ x, int64_t ld, int d,
                                                        const uint32_t *__restrict__ ids,
                                                        const long long *__restrict__ n_rows_dev,
                                                        int64_t n_rows_max, void *__restrict__ out, int64_t ld_out,
                                                        int kp, float *__restrict__ inv_norm,
                                                        float *__restrict__ scale, unsigned *status,
                                                        float *__restrict__ raw_out, int64_t raw_ld)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t n_rows = n_rows_dev ? (int64_t)*n_rows_dev : n_rows_max;
    if (n_rows > n_rows_max) n_rows = n_rows_max;
    const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    const bool raw_vec = ((raw_ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(raw_out) & 15) == 0);
    for (int64_t c = warp_global; c < n_rows; c += n_warps) {
        const int64_t r = ids ? (int64_t)ids[c] : c;
        // the raw copy keeps the source row number r
        normalize_row<FMT>(x + r * ld, d, vec, out, c, ld_out, kp, inv_norm, scale, status, lane,
                           raw_out ? raw_out + r * raw_ld : nullptr, raw_vec);
    }
}

// Batched form: the rows of many relations go to one concatenated operand.
// Global row g belongs to relation j with row_off[j] <= g < row_off[j + 1].
template <int FMT>
__global__ void __launch_bounds__(256) normalize_batch_kernel(const float *const *__restrict__ xs,
                                                              const long long *__restrict__ lds,
                                                              const long long *__restrict__ row_off, int n_rel,
                                                              int d, void *__restrict__ out, int kp,
                                                              float *__restrict__ inv_norm,
                                                              float *__restrict__ scale, unsigned *status,
                                                              const uint32_t *__restrict__ ids,
                                                              const long long *__restrict__ src_off)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = row_off[n_rel];
    for (int64_t g = warp_global; g < total; g += n_warps) {
        int lo = 0, hi = n_rel;  // row_off[lo] <= g < row_off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(row_off + mid) <= g) lo = mid;
            else hi = mid;
        }
        const float *x = xs[lo];
        const int64_t ld = lds[lo];
        const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
        const int64_t r = ids ? (int64_t)ids[g] - src_off[lo] : g - row_off[lo];
        normalize_row<FMT>(x + r * ld, d, vec, out, g, kp, kp, inv_norm, scale, status, lane);
    }
}

// Batched form for 16-byte aligned rows with d % 4 == 0 and d <= 128 V: each warp takes RW consecutive rows
// at a time and issues all their loads before reducing, so RW rows are in flight per warp; the job of a
// row is found by one search per warp, then by moving forward (a warp's rows only increase).  Sums,
// maxima, their order and the butterfly are those of normalize_row, so the outputs are bit-identical; a
// row whose plain sum of squares over- or underflows is handed to normalize_row.
template <int FMT, int V, int RW>
__global__ void __launch_bounds__(256) normalize_batch_rows_kernel(const float *const *__restrict__ xs,
                                                                   const long long *__restrict__ lds,
                                                                   const long long *__restrict__ row_off, int n_rel,
                                                                   int d, void *__restrict__ out, int kp,
                                                                   float *__restrict__ inv_norm,
                                                                   float *__restrict__ scale, unsigned *status,
                                                                   const uint32_t *__restrict__ ids,
                                                                   const long long *__restrict__ src_off)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = row_off[n_rel];
    const int d4 = d >> 2, groups = kp >> 2;
    // source row of operand row g of relation j
    auto src_row = [&](int64_t g, int j) -> int64_t {
        return ids ? (int64_t)__ldg(ids + g) - __ldg(src_off + j) : g - __ldg(row_off + j);
    };
    int job = -1;
    for (int64_t g0 = warp_global * RW; g0 < total; g0 += n_warps * RW) {
        if (job < 0) {
            int lo = 0, hi = n_rel;  // row_off[lo] <= g0 < row_off[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(row_off + mid) <= g0) lo = mid;
                else hi = mid;
            }
            job = lo;
        }
        float4 v[RW][V];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int64_t g = g0 + r;
            const float *src = nullptr;
            if (g < total) {  // warp-uniform
                while (__ldg(row_off + job + 1) <= g) ++job;
                src = xs[job] + src_row(g, job) * lds[job];
            }
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int e = lane + 32 * q;
                v[r][q] = (src && e < d4) ? __ldg(reinterpret_cast<const float4 *>(src) + e)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int64_t g = g0 + r;
            if (g >= total) break;  // warp-uniform
            float ss = 0.f, mx = 0.f;
#pragma unroll
            for (int q = 0; q < V; ++q) {
                if (lane + 32 * q < d4) {
                    ss = fmaf(v[r][q].x, v[r][q].x, ss);
                    ss = fmaf(v[r][q].y, v[r][q].y, ss);
                    ss = fmaf(v[r][q].z, v[r][q].z, ss);
                    ss = fmaf(v[r][q].w, v[r][q].w, ss);
                    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v[r][q].x), fabsf(v[r][q].y)),
                                         fmaxf(fabsf(v[r][q].z), fabsf(v[r][q].w))));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ss += __shfl_xor_sync(0xffffffffu, ss, o);
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            const bool bad = isnan(ss) || !isfinite(mx);
            if (!bad && !(isfinite(ss) && (ss >= 0x1p-100f || mx == 0.f))) {
                // over- or underflow of the plain sum: the rescaled path
                int jb = job;
                while (__ldg(row_off + jb) > g) --jb;
                normalize_row<FMT>(xs[jb] + src_row(g, jb) * lds[jb], d, true, out, g, kp, kp, inv_norm, scale,
                                   status, lane);
                continue;
            }
            const float inv = bad ? 0.f : (ss > 0.f ? 1.0f / sqrtf(ss) : 0.f);
            if (bad && lane == 0) atomicOr(status, ERR_NONFINITE);
            float rsc = 1.f;
            if (FMT == FMT_FP8) {
                const float ymax = mx * inv;
                const float sc = ymax > 0.f ? ymax / 448.f : 1.f;
                rsc = 1.0f / sc;
                if (lane == 0) scale[g] = sc;
            }
            if (lane == 0 && inv_norm) inv_norm[g] = inv;
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int e = lane + 32 * q;
                if (e >= groups) break;
                float4 y = e < d4 ? v[r][q] : make_float4(0.f, 0.f, 0.f, 0.f);
                y.x *= inv;
                y.y *= inv;
                y.z *= inv;
                y.w *= inv;
                const int k = 4 * e;
                if (FMT == FMT_F32) {
                    *reinterpret_cast<float4 *>(reinterpret_cast<float *>(out) + g * kp + k) = y;
                } else if (FMT == FMT_BF16) {
                    __nv_bfloat162 lo = __floats2bfloat162_rn(y.x, y.y);
                    __nv_bfloat162 hi = __floats2bfloat162_rn(y.z, y.w);
                    uint2 u;
                    u.x = *reinterpret_cast<uint32_t *>(&lo);
                    u.y = *reinterpret_cast<uint32_t *>(&hi);
                    *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(out) + g * kp + k) = u;
                } else {
                    const __nv_fp8x2_storage_t lo =
                        __nv_cvt_float2_to_fp8x2(make_float2(y.x * rsc, y.y * rsc), __NV_SATFINITE, __NV_E4M3);
                    const __nv_fp8x2_storage_t hi =
                        __nv_cvt_float2_to_fp8x2(make_float2(y.z * rsc, y.w * rsc), __NV_SATFINITE, __NV_E4M3);
                    *reinterpret_cast<uint32_t *>(reinterpret_cast<__nv_fp8_storage_t *>(out) + g * kp + k) =
                        (uint32_t)lo | ((uint32_t)hi << 16);
                }
            }
        }
    }
}

// e4m3 with a scale shared by each group of G consecutive output rows (the
// rows of one column tile of the contraction): scale[c] = the largest per-row
// scale max|y|/448 of c's group, so the epilogue can fold one column scale per
// tile into its threshold.  Unit rows have |y| <= 1, so every shared scale is
// still at most 1/448 and the guard band of the per-row form covers it.
__global__ void scale_group_max_kernel(float *__restrict__ scale, const long long *__restrict__ n_rows_dev,
                                       int64_t n_rows_max, int G)
{
    int64_t n = *n_rows_dev;
    if (n > n_rows_max) n = n_rows_max;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g0 = w * G; g0 < n; g0 += nw * G) {
        const int64_t g1 = g0 + G < n ? g0 + G : n;
        float m = 0.f;
        for (int64_t c = g0 + lane; c < g1; c += 32) m = fmaxf(m, scale[c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        for (int64_t c = g0 + lane; c < g1; c += 32) scale[c] = m;
    }
}

// Quantise kept row c (one warp): q = rn_satfinite(x_r * inv[c] / scale[c]) in
// e4m3, zero padded to kp.
__global__ void __launch_bounds__(256) fp8_quantize_kernel(const float *__restrict__ x, int64_t ld, int d,
                                                           const uint32_t *__restrict__ ids,
                                                           const long long *__restrict__ n_rows_dev,
                                                           int64_t n_rows_max, __nv_fp8_storage_t *__restrict__ out,
                                                           int64_t ld_out, int kp, const float *__restrict__ inv_norm,
                                                           const float *__restrict__ scale)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t n_rows = *n_rows_dev;
    if (n_rows > n_rows_max) n_rows = n_rows_max;
    const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    for (int64_t c = warp_global; c < n_rows; c += n_warps) {
        const float *src = x + (ids ? (int64_t)ids[c] : c) * ld;
        const float m = inv_norm[c] / scale[c];
        for (int g = lane; g < (kp >> 2); g += 32) {
            const int k = 4 * g;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (vec && k + 3 < d) {
                v = __ldg(reinterpret_cast<const float4 *>(src + k));
            } else {
                if (k + 0 < d) v.x = __ldg(src + k + 0);
                if (k + 1 < d) v.y = __ldg(src + k + 1);
                if (k + 2 < d) v.z = __ldg(src + k + 2);
                if (k + 3 < d) v.w = __ldg(src + k + 3);
            }
            const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v.x * m, v.y * m), __NV_SATFINITE, __NV_E4M3);
            const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v.z * m, v.w * m), __NV_SATFINITE, __NV_E4M3);
            *reinterpret_cast<uint32_t *>(out + c * ld_out + k) = (uint32_t)lo | ((uint32_t)hi << 16);
        }
    }
}

cudaError_t launch_normalize_fp8_grouped(const float *x, int64_t ld, int d, const uint32_t *ids,
                                         const long long *n_rows_dev, int64_t n_rows_max, void *out, int64_t ld_out,
                                         int kp, float *inv_norm, float *scale, int group, unsigned *status,
                                         int num_sms, cudaStream_t st, float *raw_out, int64_t raw_ld)
{
    if (n_rows_max <= 0) return cudaSuccess;
    if (!inv_norm || !scale || group < 1) return cudaErrorInvalidValue;
    int64_t blocks = (n_rows_max + 7) / 8;
    const int64_t cap = (int64_t)num_sms * 16;
    if (blocks > cap) blocks = cap;
    // norms and per-row scales, then the group maxima, then the quantised rows
    normalize_kernel<FMT_FP8><<<(unsigned)blocks, 256, 0, st>>>(x, ld, d, ids, n_rows_dev, n_rows_max, nullptr,
                                                                ld_out, kp, inv_norm, scale, status, raw_out,
                                                                raw_ld);
    int64_t gblocks = ((n_rows_max + group - 1) / group + 7) / 8;
    if (gblocks > cap) gblocks = cap;
    if (gblocks < 1) gblocks = 1;
    scale_group_max_kernel<<<(unsigned)gblocks, 256, 0, st>>>(scale, n_rows_dev, n_rows_max, group);
    // the second read of the rows comes from the raw copy when there is one
    fp8_quantize_kernel<<<(unsigned)blocks, 256, 0, st>>>(raw_out ? raw_out : x, raw_out ? raw_ld : ld, d, ids,
                                                          n_rows_dev, n_rows_max,
                                                          reinterpret_cast<__nv_fp8_storage_t *>(out), ld_out, kp,
                                                          inv_norm, scale);
    return cudaGetLastError();
}

cudaError_t launch_sel_count(const SelArgs &s, int64_t n, uint32_t *block_counts, cudaStream_t st)
{
    const int64_t nb = (n + SEL_ROWS_PER_BLOCK - 1) / SEL_ROWS_PER_BLOCK;
    if (nb == 0) return cudaSuccess;
    sel_count_kernel<<<(unsigned)nb, SEL_THREADS, 0, st>>>(s, n, block_counts);
    return cudaGetLastError();
}

cudaError_t launch_sel_scan(const uint32_t *block_counts, int64_t n_blocks, uint32_t *block_offsets,
                            long long *n_sel, cudaStream_t st)
{
    sel_scan_kernel<<<1, 1024, 0, st>>>(block_counts, n_blocks, block_offsets, n_sel);
    return cudaGetLastError();
}

cudaError_t launch_sel_scatter(const SelArgs &s, int64_t n, const uint32_t *block_offsets, uint32_t *ids,
                               cudaStream_t st)
{
    const int64_t nb = (n + SEL_ROWS_PER_BLOCK - 1) / SEL_ROWS_PER_BLOCK;
    if (nb == 0) return cudaSuccess;
    sel_scatter_kernel<<<(unsigned)nb, SEL_THREADS, 0, st>>>(s, n, block_offsets, ids);
    return cudaGetLastError();
}

cudaError_t launch_set_count(long long *n_sel, long long value, cudaStream_t st)
{
    set_count_kernel<<<1, 1, 0, st>>>(n_sel, value);
    return cudaGetLastError();
}

cudaError_t launch_normalize(int fmt, const float *x, int64_t ld, int d, const uint32_t *ids,
                             const long long *n_rows_dev, int64_t n_rows_max, void *out, int64_t ld_out, int kp,
                             float *inv_norm, float *scale, unsigned *status, int num_sms, cudaStream_t st,
                             float *raw_out, int64_t raw_ld)
{
    if (n_rows_max <= 0) return cudaSuccess;
    // 8 warps per block, up to 16 blocks per SM, grid-stride over rows
    int64_t blocks = (n_rows_max + 7) / 8;
    const int64_t cap = (int64_t)num_sms * 16;
    if (blocks > cap) blocks = cap;
    switch (fmt) {
    case FMT_F32:
        normalize_kernel<FMT_F32><<<(unsigned)blocks, 256, 0, st>>>(x, ld, d, ids, n_rows_dev, n_rows_max, out,
                                                                    ld_out, kp, inv_norm, scale, status, raw_out, raw_ld);
        break;
    case FMT_BF16:
        normalize_kernel<FMT_BF16><<<(unsigned)blocks, 256, 0, st>>>(x, ld, d, ids, n_rows_dev, n_rows_max, out,
                                                                     ld_out, kp, inv_norm, scale, status, raw_out, raw_ld);
        break;
    case FMT_FP8:
        normalize_kernel<FMT_FP8><<<(unsigned)blocks, 256, 0, st>>>(x, ld, d, ids, n_rows_dev, n_rows_max, out,
                                                                    ld_out, kp, inv_norm, scale, status, raw_out, raw_ld);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int FMT, int V>
static void launch_batch_rows(int64_t total_rows, const float *const *xs, const long long *lds,
                              const long long *row_off, int n_rel, int d, void *out, int kp, float *inv_norm,
                              float *scale, unsigned *status, int num_sms, cudaStream_t st, const uint32_t *ids,
                              const long long *src_off)
{
    constexpr int RW = V <= 4 ? 4 : 2;
    // one wave of resident blocks walks the rows (a second wave would start only after the first ended)
    static int per_sm = 0;
    if (per_sm == 0 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, normalize_batch_rows_kernel<FMT, V, RW>, 256, 0) !=
            cudaSuccess)
        per_sm = 1;
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (total_rows + 8 * RW - 1) / (8 * RW);
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    normalize_batch_rows_kernel<FMT, V, RW><<<(unsigned)blocks, 256, 0, st>>>(xs, lds, row_off, n_rel, d, out, kp,
                                                                              inv_norm, scale, status, ids, src_off);
}

template <int FMT>
static cudaError_t launch_batch_rows_d(int64_t total_rows, const float *const *xs, const long long *lds,
                                       const long long *row_off, int n_rel, int d, void *out, int kp,
                                       float *inv_norm, float *scale, unsigned *status, int num_sms, cudaStream_t st,
                                       const uint32_t *ids, const long long *src_off)
{
#define EJ_NB_ARGS total_rows, xs, lds, row_off, n_rel, d, out, kp, inv_norm, scale, status, num_sms, st, ids, src_off
    if (d <= 128) launch_batch_rows<FMT, 1>(EJ_NB_ARGS);
    else if (d <= 256) launch_batch_rows<FMT, 2>(EJ_NB_ARGS);
    else if (d <= 384) launch_batch_rows<FMT, 3>(EJ_NB_ARGS);
    else if (d <= 512) launch_batch_rows<FMT, 4>(EJ_NB_ARGS);
    else if (d <= 768) launch_batch_rows<FMT, 6>(EJ_NB_ARGS);
    else launch_batch_rows<FMT, 8>(EJ_NB_ARGS);
#undef EJ_NB_ARGS
    return cudaGetLastError();
}

cudaError_t launch_normalize_batch(int fmt, const float *const *xs, const long long *lds, const long long *row_off,
                                   int n_rel, int64_t total_rows, int d, void *out, int kp, float *inv_norm,
                                   float *scale, unsigned *status, int num_sms, cudaStream_t st, bool aligned,
                                   const uint32_t *ids, const long long *src_off)
{
    if (total_rows <= 0) return cudaSuccess;
    if (aligned && d % 4 == 0 && d <= 1024 && kp <= 4 * 32 * ((d + 127) / 128)) {
        // every relation's rows start on 16 bytes (checked by the host)
        switch (fmt) {
        case FMT_F32:
            return launch_batch_rows_d<FMT_F32>(total_rows, xs, lds, row_off, n_rel, d, out, kp, inv_norm, scale,
                                                status, num_sms, st, ids, src_off);
        case FMT_BF16:
            return launch_batch_rows_d<FMT_BF16>(total_rows, xs, lds, row_off, n_rel, d, out, kp, inv_norm, scale,
                                                 status, num_sms, st, ids, src_off);
        case FMT_FP8:
            return launch_batch_rows_d<FMT_FP8>(total_rows, xs, lds, row_off, n_rel, d, out, kp, inv_norm, scale,
                                                status, num_sms, st, ids, src_off);
        default: return cudaErrorInvalidValue;
        }
    }
    int64_t blocks = (total_rows + 7) / 8;
    const int64_t cap = (int64_t)num_sms * 16;
    if (blocks > cap) blocks = cap;
    switch (fmt) {
    case FMT_F32:
        normalize_batch_kernel<FMT_F32><<<(unsigned)blocks, 256, 0, st>>>(xs, lds, row_off, n_rel, d, out, kp,
                                                                          inv_norm, scale, status, ids, src_off);
        break;
    case FMT_BF16:
        normalize_batch_kernel<FMT_BF16><<<(unsigned)blocks, 256, 0, st>>>(xs, lds, row_off, n_rel, d, out, kp,
                                                                           inv_norm, scale, status, ids, src_off);
        break;
    case FMT_FP8:
        normalize_batch_kernel<FMT_FP8><<<(unsigned)blocks, 256, 0, st>>>(xs, lds, row_off, n_rel, d, out, kp,
                                                                          inv_norm, scale, status, ids, src_off);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ej
