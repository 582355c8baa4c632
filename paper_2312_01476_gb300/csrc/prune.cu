// Learned tile pruning: reorder rows so that tiles are coherent in sketch
// space, bound the sketch cosine of every tile pair, keep the tile pairs that
// can hold a match.  The contraction then runs on the kept tile pairs only
// and every candidate is re-scored exactly, so pruning can only lose pairs
// whose sketch cosine falls below the calibrated sketch threshold.
//
// Tile bound: with unit centroid c_T and angular radius rho_T (largest angle
// between c_T and a member sketch), any pair (a in A, b in B) satisfies
//   angle(s_a, s_b) >= angle(c_A, c_B) - rho_A - rho_B
// (triangle inequality for angles on the sphere), hence
//   cos(s_a, s_b) <= cos(max(0, angle(c_A, c_B) - rho_A - rho_B)).
#include <algorithm>
#include <cfloat>

#include "mlp_internal.cuh"

namespace ej {

namespace {
constexpr int SK = 64;          // sketch width handled by these kernels
constexpr float RADIUS_MARGIN = 2e-3f;  // radians, covers FP32 rounding of dots near 1
constexpr int NB = PRUNE_BALLS;
}  // namespace

// One thread per row: nearest anchor (largest dot) among the row's group's anchors.
__global__ void assign_keys_kernel(const float *__restrict__ S, int64_t n, const float *__restrict__ anchors,
                                   int n_anchor, const uint32_t *__restrict__ grp, uint32_t *__restrict__ key)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[SK];
#pragma unroll
    for (int q = 0; q < SK / 4; ++q) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(S + r * SK) + q);
        x[4 * q] = v.x;
        x[4 * q + 1] = v.y;
        x[4 * q + 2] = v.z;
        x[4 * q + 3] = v.w;
    }
    const uint32_t g = grp ? grp[r] : 0u;
    const float *an = anchors + (int64_t)g * n_anchor * SK;
    float best = -FLT_MAX;
    int bi = 0;
    for (int a = 0; a < n_anchor; ++a) {
        float dot = 0.f;
#pragma unroll
        for (int q = 0; q < SK / 4; ++q) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(an + (int64_t)a * SK) + q);
            dot = fmaf(x[4 * q], v.x, dot);
            dot = fmaf(x[4 * q + 1], v.y, dot);
            dot = fmaf(x[4 * q + 2], v.z, dot);
            dot = fmaf(x[4 * q + 3], v.w, dot);
        }
        if (dot > best) {
            best = dot;
            bi = a;
        }
    }
    key[r] = g * (uint32_t)n_anchor + (uint32_t)bi;
}

__global__ void key_histogram_kernel(const uint32_t *__restrict__ key, int64_t n, uint32_t *__restrict__ hist)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(hist + key[r], 1u);
}

__global__ void __launch_bounds__(1024) key_scan_kernel(uint32_t *h, int nk)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nk; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nk ? h[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const uint32_t excl = carry + (warp ? warp_tot[warp - 1] : 0u) + x - v;
        __syncthreads();
        if (i < nk) h[i] = excl;
        if (threadIdx.x == 0) carry += warp_tot[31];
        __syncthreads();
    }
}

__global__ void key_scatter_kernel(const uint32_t *__restrict__ key, int64_t n, uint32_t *__restrict__ cursor,
                                   uint32_t *__restrict__ perm)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        perm[atomicAdd(cursor + key[r], 1u)] = (uint32_t)r;
}

// One warp per output row: 16-byte copies (row_bytes is a multiple of 16).
__global__ void gather_rows_kernel(const uint4 *__restrict__ in, int64_t row_u4, const uint32_t *__restrict__ perm,
                                   int64_t n, uint4 *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < n; i += nw) {
        const uint4 *src = in + (int64_t)perm[i] * row_u4;
        uint4 *dst = out + i * row_u4;
        for (int64_t q = lane; q < row_u4; q += 32) dst[q] = __ldg(src + q);
    }
}

__global__ void gather_u32_kernel(const uint32_t *__restrict__ in, const uint32_t *__restrict__ perm, int64_t n,
                                  uint32_t *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

__global__ void gather_f32_kernel(const float *__restrict__ in, const uint32_t *__restrict__ perm, int64_t n,
                                  float *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

// Covering anchors (the reorder of the pruned join).  Rows are grouped by the
// anchor they are most similar to in sketch space; for the groups to be
// coherent, every group of mutually similar rows needs an anchor of its own
// (with fewer anchors than groups, nearest-anchor assignment splits groups
// between unrelated anchors).  Anchors are therefore drawn, in rounds, from
// the rows of a sample that no anchor covers yet (cosine >= tau), in a fixed
// pseudo-random order; a candidate covered by an earlier candidate of the
// same round is dropped, so that each group gets about one anchor.

// drop[a] = 1 when some earlier candidate b < a has <S[cand[a]], S[cand[b]]> >= tau
// (one warp per candidate).
__global__ void cover_drop_kernel(const float *__restrict__ S, const uint32_t *__restrict__ cand, int nc, float tau,
                                  unsigned char *__restrict__ drop)
{
    // one warp per candidate a; its lanes test 32 earlier candidates at a time, each lane a full 64-term dot
    const int lane = threadIdx.x & 31;
    const int a = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (a >= nc) return;
    float x[SK];
    const float4 *xa = reinterpret_cast<const float4 *>(S + (int64_t)cand[a] * SK);
#pragma unroll
    for (int q = 0; q < SK / 4; ++q) {
        const float4 v = __ldg(xa + q);
        x[4 * q] = v.x;
        x[4 * q + 1] = v.y;
        x[4 * q + 2] = v.z;
        x[4 * q + 3] = v.w;
    }
    bool hit = false;
    for (int b0 = 0; b0 < a; b0 += 32) {
        const int b = b0 + lane;
        if (b < a) {
            const float4 *yb = reinterpret_cast<const float4 *>(S + (int64_t)cand[b] * SK);
            float dot = 0.f;
#pragma unroll
            for (int q = 0; q < SK / 4; ++q) {
                const float4 v = __ldg(yb + q);
                dot = fmaf(x[4 * q], v.x, dot);
                dot = fmaf(x[4 * q + 1], v.y, dot);
                dot = fmaf(x[4 * q + 2], v.z, dot);
                dot = fmaf(x[4 * q + 3], v.w, dot);
            }
            hit = dot >= tau;
        }
        if (__any_sync(0xffffffffu, hit)) {
            hit = true;
            break;
        }
    }
    if (lane == 0) drop[a] = hit ? 1 : 0;
}

// covered[r] = 1 for every candidate (r, anchor) of a threshold contraction of the sample rows against
// the round's anchors.
__global__ void cover_mark_kernel(const uint2 *__restrict__ cand, const unsigned long long *__restrict__ count,
                                  uint64_t cap, unsigned char *__restrict__ covered)
{
    uint64_t n = *count;
    if (n > cap) n = cap;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x)
        covered[cand[t].x] = 1;
}

// One block (256 threads) per tile of tile_rows (<= 256) consecutive sketch
// rows (in reorder order).  The tile is described by up to NB balls (see
// below); any assignment of rows to balls gives a valid bound, this one keeps
// the balls small when the tile holds up to NB well-separated groups.  Ball = unit centroid + angular radius (largest
// angle between the centroid and a member, plus a rounding margin); unused
// balls get radius -1.
// Balls of one tile (a block per tile of tile_rows <= 256 sketch rows): NB seeds by farthest-point sampling
// (the first row, then the row least similar to the seeds so far, ties to the smaller row), every row joins
// its most similar seed (ties to the earlier seed), and each ball is the unit centroid of its rows with the
// angular radius that covers them (RADIUS_MARGIN added; -1: unused ball).  The tile's rows are staged in
// shared memory (rows padded to SK + 1 floats, so that the lanes' rows fall in distinct banks) and every
// warp takes part; the dot products are the per-row FMA chains over q in order.
constexpr int TS_LD = SK + 1;

__device__ __forceinline__ float row_dot(const float *x, const float *y)
{
    float dot = 0.f;
#pragma unroll 16
    for (int q = 0; q < SK; ++q) dot = fmaf(x[q], y[q], dot);
    return dot;
}

__global__ void __launch_bounds__(256) tile_stats_kernel(const float *__restrict__ S, int64_t n, int tile_rows,
                                                         float *__restrict__ centroid, float *__restrict__ radius)
{
    extern __shared__ float xs[];  // [tile_rows][TS_LD]
    __shared__ float c[NB][SK];
    __shared__ int run_of[256];
    __shared__ float maxd[256];
    __shared__ int seeds[NB];
    __shared__ int cnt[NB];
    __shared__ float wv[8];
    __shared__ int wi[8];
    const int64_t r0 = (int64_t)blockIdx.x * tile_rows;
    int64_t r1 = r0 + tile_rows;
    if (r1 > n) r1 = n;
    const int rows = (int)(r1 - r0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < rows * SK; e += blockDim.x) xs[(e / SK) * TS_LD + e % SK] = S[r0 * SK + e];
    for (int e = tid; e < NB * SK; e += blockDim.x) c[e / SK][e % SK] = 0.f;
    if (tid < NB) cnt[tid] = 0;
    __syncthreads();
    // farthest-point seeds
    int seed = 0;
    for (int j = 0; j < NB; ++j) {
        if (tid == 0) seeds[j] = seed;
        float bv = 3.f;
        int bi = 0x7fffffff;
        if (tid < rows) {
            const float dot = row_dot(xs + tid * TS_LD, xs + seed * TS_LD);
            const float m = j == 0 ? dot : fmaxf(maxd[tid], dot);
            maxd[tid] = m;
            bv = m;
            bi = tid;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov < bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            wv[warp] = bv;
            wi[warp] = bi;
        }
        __syncthreads();
        bv = wv[0];
        bi = wi[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (wv[w] < bv || (wv[w] == bv && wi[w] < bi)) {
                bv = wv[w];
                bi = wi[w];
            }
        seed = bi;
        __syncthreads();
    }
    if (tid < rows) {
        const float *x = xs + tid * TS_LD;
        float best = -3.f;
        int bb = 0;
        for (int j = 0; j < NB; ++j) {
            const float dot = row_dot(x, xs + seeds[j] * TS_LD);
            if (dot > best) {
                best = dot;
                bb = j;
            }
        }
        run_of[tid] = bb;
    }
    __syncthreads();
    // centroid sums: one thread per (ball, dim), looping over the tile's rows
    for (int e = tid; e < NB * SK; e += blockDim.x) {
        const int bl = e / SK, q = e % SK;
        float acc = 0.f;
        int k = 0;
        for (int r = 0; r < rows; ++r)
            if (run_of[r] == bl) {
                acc += xs[r * TS_LD + q];
                ++k;
            }
        c[bl][q] = acc;
        if (q == 0) cnt[bl] = k;
    }
    __syncthreads();
    if (warp < NB) {
        float ss = c[warp][lane] * c[warp][lane] + c[warp][lane + 32] * c[warp][lane + 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
        c[warp][lane] *= inv;
        c[warp][lane + 32] *= inv;
    }
    __syncthreads();
    // the smallest cosine between a ball's centroid and its members: one warp per ball
    if (warp < NB) {
        float mn = 1.f;
        for (int r = lane; r < rows; r += 32) {
            if (run_of[r] != warp) continue;
            float dot = 0.f;
#pragma unroll 16
            for (int q = 0; q < SK; ++q) dot = fmaf(c[warp][q], xs[r * TS_LD + q], dot);
            mn = fminf(mn, dot);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        if (lane == 0) {
            float ss = 0.f;
            for (int q = 0; q < SK; ++q) ss += c[warp][q] * c[warp][q];
            float rad;
            if (cnt[warp] == 0) rad = -1.f;                   // unused ball
            else if (ss < 0.5f) rad = 3.14159265f;             // degenerate centroid bounds nothing
            else rad = acosf(fmaxf(-1.f, fminf(1.f, mn))) + RADIUS_MARGIN;
            radius[(int64_t)blockIdx.x * NB + warp] = rad;
        }
    }
    for (int e = tid; e < NB * SK; e += blockDim.x)
        centroid[(int64_t)blockIdx.x * NB * SK + e] = c[e / SK][e % SK];
}

// TP x TP tile pairs per block (256 threads, 2 x 2 pairs each).  A tile pair is kept when some ball pair
// (a, b) has cos(max(0, angle(c_a, c_b) - r_a - r_b)) >= cos_keep, i.e. angle(c_a, c_b) <= r_a + r_b + alpha
// with alpha = acos(cos_keep): always when r_a + alpha + r_b >= pi, else when
// c_a . c_b >= cos(r_a + alpha) cos(r_b) - sin(r_a + alpha) sin(r_b) (= cos(r_a + alpha + r_b)), tested with
// a margin of 1e-6 towards keeping.  The 64-term dots of a thread's 8 x 8 ball pairs are register-tiled;
// the balls sit in shared memory ball-major ([ball][tile]), so a warp's loads fall on distinct banks.
// Kept pairs are appended with one atomic per warp.
constexpr int TP = 32;
constexpr float PI_F = 3.14159265358979f;
__global__ void __launch_bounds__(256) tile_pairs_kernel(const float *__restrict__ cA, const float *__restrict__ rA,
                                                         int64_t tA, const float *__restrict__ cB,
                                                         const float *__restrict__ rB, int64_t tB, float cos_keep,
                                                         uint2 *__restrict__ list, uint64_t cap,
                                                         unsigned long long *count, int sym)
{
    extern __shared__ float sm[];
    float *sa = sm;                       // [NB][TP][SK + 1]: ball x of tile t at row x * TP + t
    float *sb = sa + NB * TP * (SK + 1);  // [NB][TP][SK + 1]
    float *pa = sb + NB * TP * (SK + 1);  // [NB * TP][3]: r, cos(r + alpha), sin(r + alpha)
    float *pb = pa + NB * TP * 3;         // [NB * TP][3]: r, cos r, sin r
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t a0 = (int64_t)blockIdx.y * TP, b0 = (int64_t)blockIdx.x * TP;
    const float alpha = cos_keep >= 1.f ? 0.f : (cos_keep <= -1.f ? PI_F : acosf(cos_keep));
    for (int e = tid; e < TP * NB * SK; e += 256) {
        const int tb = e / SK, q = e % SK;  // tb = tile * NB + ball in the global order
        const int t = tb / NB, x = tb % NB;
        sa[(x * TP + t) * (SK + 1) + q] = a0 + t < tA ? cA[((a0 + t) * NB + x) * SK + q] : 0.f;
        sb[(x * TP + t) * (SK + 1) + q] = b0 + t < tB ? cB[((b0 + t) * NB + x) * SK + q] : 0.f;
    }
    for (int e = tid; e < TP * NB; e += 256) {
        const int t = e / NB, x = e % NB, k = x * TP + t;
        const float ra = a0 + t < tA ? rA[(a0 + t) * NB + x] : -1.f;
        const float rb = b0 + t < tB ? rB[(b0 + t) * NB + x] : -1.f;
        pa[3 * k] = ra;
        pa[3 * k + 1] = cosf(ra + alpha);
        pa[3 * k + 2] = sinf(ra + alpha);
        pb[3 * k] = rb;
        pb[3 * k + 1] = cosf(rb);
        pb[3 * k + 2] = sinf(rb);
    }
    __syncthreads();
    // thread -> 2 x 2 tile pairs: rows 2 ty + i, cols 2 tx + j (ty, tx in 0..15), i.e. 8 x 8 ball pairs
    const int ty = tid >> 4, tx = tid & 15;
    float acc[2][NB][2][NB];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int x = 0; x < NB; ++x)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int y = 0; y < NB; ++y) acc[i][x][j][y] = 0.f;
#pragma unroll 4
    for (int q = 0; q < SK; ++q) {
        float av[2][NB], bv[2][NB];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int x = 0; x < NB; ++x) av[i][x] = sa[(x * TP + 2 * ty + i) * (SK + 1) + q];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int y = 0; y < NB; ++y) bv[j][y] = sb[(y * TP + 2 * tx + j) * (SK + 1) + q];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int x = 0; x < NB; ++x)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int y = 0; y < NB; ++y) acc[i][x][j][y] = fmaf(av[i][x], bv[j][y], acc[i][x][j][y]);
    }
    unsigned mask = 0u;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int ta = 2 * ty + i;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int tb = 2 * tx + j;
            if (a0 + ta >= tA || b0 + tb >= tB) continue;
            if (sym && ((a0 + ta) >> 1) > b0 + tb) continue;  // self-join: block pairs on or above the diagonal
            bool keep = false;
#pragma unroll
            for (int x = 0; x < NB; ++x) {
                const float *qa = pa + 3 * (x * TP + ta);
#pragma unroll
                for (int y = 0; y < NB; ++y) {
                    const float *qb = pb + 3 * (y * TP + tb);
                    if (qa[0] < 0.f || qb[0] < 0.f) continue;  // unused ball
                    if (qa[0] + alpha + qb[0] >= PI_F)
                        keep = true;
                    else
                        keep |= acc[i][x][j][y] >= qa[1] * qb[1] - qa[2] * qb[2] - 1e-6f;
                }
            }
            if (keep) mask |= 1u << (i * 2 + j);
        }
    }
    const int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    if (tot == 0) return;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(count, (unsigned long long)tot);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned long long p = base + (unsigned long long)(incl - cnt);
    while (mask) {
        const int b = __ffs(mask) - 1;
        mask &= mask - 1u;
        if (p < cap) list[p] = make_uint2((uint32_t)(a0 + ty * 2 + (b >> 1)), (uint32_t)(b0 + tx * 2 + (b & 1)));
        ++p;
    }
}

static unsigned grid_for(int64_t n, int per_block)
{
    int64_t b = (n + per_block - 1) / per_block;
    if (b > 65535 * 16) b = 65535 * 16;
    return (unsigned)std::max<int64_t>(b, 1);
}

cudaError_t launch_assign_keys(const float *S, int64_t n, int k, const float *anchors, int n_anchor,
                               const uint32_t *grp, uint32_t *key, int num_sms, cudaStream_t st)
{
    (void)num_sms;
    if (k != SK) return cudaErrorInvalidValue;
    if (n <= 0) return cudaSuccess;
    assign_keys_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(S, n, anchors, n_anchor, grp, key);
    return cudaGetLastError();
}

cudaError_t launch_key_histogram(const uint32_t *key, int64_t n, uint32_t *hist, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    key_histogram_kernel<<<grid_for(n, 256 * 8), 256, 0, st>>>(key, n, hist);
    return cudaGetLastError();
}

cudaError_t launch_key_scan(uint32_t *hist, int n_keys, cudaStream_t st)
{
    key_scan_kernel<<<1, 1024, 0, st>>>(hist, n_keys);
    return cudaGetLastError();
}

cudaError_t launch_key_scatter(const uint32_t *key, int64_t n, uint32_t *cursor, uint32_t *perm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    key_scatter_kernel<<<grid_for(n, 256 * 8), 256, 0, st>>>(key, n, cursor, perm);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const void *in, int64_t row_bytes, const uint32_t *perm, int64_t n, void *out,
                               cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (row_bytes % 16) return cudaErrorInvalidValue;
    gather_rows_kernel<<<grid_for(n, 8), 256, 0, st>>>((const uint4 *)in, row_bytes / 16, perm, n, (uint4 *)out);
    return cudaGetLastError();
}

cudaError_t launch_gather_u32(const uint32_t *in, const uint32_t *perm, int64_t n, uint32_t *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    gather_u32_kernel<<<grid_for(n, 256 * 4), 256, 0, st>>>(in, perm, n, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_f32(const float *in, const uint32_t *perm, int64_t n, float *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    gather_f32_kernel<<<grid_for(n, 256 * 4), 256, 0, st>>>(in, perm, n, out);
    return cudaGetLastError();
}

cudaError_t launch_cover_drop(const float *S, const uint32_t *cand, int nc, float tau, unsigned char *drop,
                              cudaStream_t st)
{
    if (nc <= 0) return cudaSuccess;
    cover_drop_kernel<<<(unsigned)((nc + 7) / 8), 256, 0, st>>>(S, cand, nc, tau, drop);
    return cudaGetLastError();
}

cudaError_t launch_cover_mark(const uint2 *cand, const unsigned long long *count, uint64_t cap,
                              unsigned char *covered, int num_sms, cudaStream_t st)
{
    if (cap == 0) return cudaSuccess;
    const uint64_t want = (cap + 255) / 256, lim = (uint64_t)num_sms * 8;
    cover_mark_kernel<<<(unsigned)(want < lim ? (want ? want : 1) : lim), 256, 0, st>>>(cand, count, cap, covered);
    return cudaGetLastError();
}

cudaError_t launch_tile_stats(const float *S, int64_t n, int k, int tile_rows, float *centroid, float *radius,
                              cudaStream_t st)
{
    if (k != SK || tile_rows > 256) return cudaErrorInvalidValue;
    const int64_t tiles = (n + tile_rows - 1) / tile_rows;
    if (tiles <= 0) return cudaSuccess;
    const int smem = tile_rows * TS_LD * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(tile_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 * TS_LD * 4);
    if (e != cudaSuccess) return e;
    tile_stats_kernel<<<(unsigned)tiles, 256, smem, st>>>(S, n, tile_rows, centroid, radius);
    return cudaGetLastError();
}

cudaError_t launch_tile_pairs(const float *cA, const float *rA, int64_t tA, const float *cB, const float *rB,
                              int64_t tB, int k, float eps_sketch, uint2 *list, uint64_t cap,
                              unsigned long long *count, cudaStream_t st, int sym)
{
    if (k != SK) return cudaErrorInvalidValue;
    if (tA <= 0 || tB <= 0) return cudaSuccess;
    const int smem = (2 * TP * NB * (SK + 1) + 2 * TP * NB * 3) * 4;
    cudaError_t e = cudaFuncSetAttribute(tile_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((tB + TP - 1) / TP), (unsigned)((tA + TP - 1) / TP));
    tile_pairs_kernel<<<grid, 256, smem, st>>>(cA, rA, tA, cB, rB, tB, eps_sketch, list, cap, count, sym);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------------
// Tile-pair bounds on the tensor cores.  The bound of a ball pair (unit centroids c_a, c_b, angular radii
// r_a, r_b) keeps it when angle(c_a, c_b) <= r_a + alpha + r_b, alpha = acos(eps_sketch).  With
// u = r_a + alpha < pi/2 and r_b < pi/2 that is cos(angle) >= cos(u + r_b) = cos u cos r_b - sin u sin r_b,
// i.e. the dot product of the augmented rows  a = [c_a, -cos u, sin u, 0, 1, 0, 1]  and
// b = [c_b, cos r_b, sin r_b, 1, 0, 1, 0]  is >= 0.  The last four columns make the other cases exact:
// a "wide" ball (u >= pi/2, resp. r_b >= pi/2) has a zero centroid part and a 1 that meets a 1 of every
// used ball of the other side (kept with all of them, a superset of the angle test), and an unused ball
// carries -4 against a 1 of every ball of the other side (never kept).  Rows have BALL_K = 96 FP32 columns
// (70 used, zero padding): the TF32 threshold contraction of the two ball matrices at -margin then lists
// every kept ball pair.
constexpr int BALL_K = 96;

__global__ void ball_rows_kernel(const float *__restrict__ cent, const float *__restrict__ rad, int64_t n_balls,
                                 int64_t rows_pad, float alpha, int side, float *__restrict__ out)
{
    // one warp per ball row (rows beyond n_balls are zero padding)
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w0; k < rows_pad; k += nw) {
        float *o = out + k * BALL_K;
        const float r = k < n_balls ? rad[k] : -1.f;
        const bool used = r >= 0.f;
        const float u = side == 0 ? r + alpha : r;
        const bool wide = used && u >= 0.5f * PI_F;
        const bool normal = used && !wide;
        for (int q = lane; q < BALL_K; q += 32) {
            float v = 0.f;
            if (q < SK) {
                v = normal ? cent[k * SK + q] : 0.f;
            } else if (side == 0) {
                switch (q) {
                case SK: v = normal ? -cosf(u) : 0.f; break;
                case SK + 1: v = normal ? sinf(u) : 0.f; break;
                case SK + 2: v = wide ? 1.f : 0.f; break;
                case SK + 3: v = used ? 1.f : 0.f; break;
                case SK + 4: v = used ? 0.f : -4.f; break;
                case SK + 5: v = 1.f; break;
                default: break;
                }
            } else {
                switch (q) {
                case SK: v = normal ? cosf(u) : 0.f; break;
                case SK + 1: v = normal ? sinf(u) : 0.f; break;
                case SK + 2: v = used ? 1.f : 0.f; break;
                case SK + 3: v = wide ? 1.f : 0.f; break;
                case SK + 4: v = 1.f; break;
                case SK + 5: v = used ? 0.f : -4.f; break;
                default: break;
                }
            }
            o[q] = v;
        }
    }
}

// bit (ta * tB + tb) for each kept ball pair (ball rows a, b: tiles a / NB, b / NB); sym: only block pairs on
// or above the diagonal (ta / 2 <= tb)
__global__ void ball_pairs_bitmap_kernel(const uint2 *__restrict__ cand, const unsigned long long *__restrict__ count,
                                         uint64_t cap, int64_t tA, int64_t tB, int sym, uint32_t *bits)
{
    uint64_t n = *count;
    if (n > cap) n = cap;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const int64_t ta = cand[k].x / NB, tb = cand[k].y / NB;
        if (ta >= tA || tb >= tB || (sym && (ta >> 1) > tb)) continue;
        const uint64_t b = (uint64_t)ta * (uint64_t)tB + (uint64_t)tb;
        atomicOr(bits + (b >> 5), 1u << (b & 31));
    }
}

// row_cnt[ta] = kept tile pairs of A tile ta (one warp per row of the bitmap)
__global__ void bitmap_row_count_kernel(const uint32_t *__restrict__ bits, int64_t tA, int64_t tB, uint32_t *row_cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ta = w0; ta < tA; ta += nw) {
        uint32_t c = 0;
        const uint64_t b0 = (uint64_t)ta * (uint64_t)tB;
        for (int64_t tb = lane; tb < tB; tb += 32) {
            const uint64_t b = b0 + (uint64_t)tb;
            c += (bits[b >> 5] >> (b & 31)) & 1u;
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0) row_cnt[ta] = c;
    }
}

// one block: exclusive scan of the row counts in place; *count = total
__global__ void __launch_bounds__(1024) bitmap_row_scan_kernel(uint32_t *row_cnt, int64_t tA,
                                                              unsigned long long *count)
{
    __shared__ uint32_t w[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < tA; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        const uint32_t v = i < tA ? row_cnt[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t a = w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, a, o);
                if (lane >= o) a += y;
            }
            w[lane] = a;
        }
        __syncthreads();
        if (i < tA) row_cnt[i] = (uint32_t)carry + (warp ? w[warp - 1] : 0u) + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += w[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = carry;
}

// list[row_off[ta] + rank] = (ta, tb) for the set bits of row ta, in ascending tb (one warp per row)
__global__ void bitmap_row_write_kernel(const uint32_t *__restrict__ bits, int64_t tA, int64_t tB,
                                        const uint32_t *__restrict__ row_off, uint2 *__restrict__ list, uint64_t cap)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ta = w0; ta < tA; ta += nw) {
        uint64_t pos = row_off[ta];
        const uint64_t b0 = (uint64_t)ta * (uint64_t)tB;
        for (int64_t t0 = 0; t0 < tB; t0 += 32) {
            const int64_t tb = t0 + lane;
            bool set = false;
            if (tb < tB) {
                const uint64_t b = b0 + (uint64_t)tb;
                set = (bits[b >> 5] >> (b & 31)) & 1u;
            }
            const unsigned m = __ballot_sync(0xffffffffu, set);
            if (set) {
                const uint64_t p = pos + __popc(m & ((1u << lane) - 1u));
                if (p < cap) list[p] = make_uint2((uint32_t)ta, (uint32_t)tb);
            }
            pos += __popc(m);
        }
    }
}

int ball_k() { return BALL_K; }

cudaError_t launch_ball_rows(const float *cent, const float *rad, int64_t n_balls, int64_t rows_pad,
                             float eps_sketch, int side, float *out, int num_sms, cudaStream_t st)
{
    const float alpha = eps_sketch >= 1.f ? 0.f : (eps_sketch <= -1.f ? PI_F : acosf(eps_sketch));
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((rows_pad + 7) / 8, (int64_t)num_sms * 16));
    ball_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(cent, rad, n_balls, rows_pad, alpha, side, out);
    return cudaGetLastError();
}

cudaError_t launch_ball_pairs_to_list(const uint2 *cand, const unsigned long long *cand_count, uint64_t cand_cap,
                                      int64_t tA, int64_t tB, int sym, uint32_t *bits, uint32_t *row_cnt,
                                      uint2 *list, uint64_t list_cap, unsigned long long *list_count, int num_sms,
                                      cudaStream_t st)
{
    const uint64_t words = ((uint64_t)tA * (uint64_t)tB + 31) / 32;
    cudaError_t e = cudaMemsetAsync(bits, 0, words * 4, st);
    if (e != cudaSuccess) return e;
    const unsigned gc = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((cand_cap + 255) / 256, (uint64_t)num_sms * 8));
    ball_pairs_bitmap_kernel<<<gc, 256, 0, st>>>(cand, cand_count, cand_cap, tA, tB, sym, bits);
    const unsigned gr = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tA + 7) / 8, (int64_t)num_sms * 16));
    bitmap_row_count_kernel<<<gr, 256, 0, st>>>(bits, tA, tB, row_cnt);
    bitmap_row_scan_kernel<<<1, 1024, 0, st>>>(row_cnt, tA, list_count);
    bitmap_row_write_kernel<<<gr, 256, 0, st>>>(bits, tA, tB, row_cnt, list, list_cap);
    return cudaGetLastError();
}

}  // namespace ej

namespace ej {

// Argmax over the (row, anchor) candidates of the assignment contraction: the
// exact FP32 sketch cosine of each candidate, packed above the anchor index,
// kept per row with a 64-bit atomicMax (the candidates' cosines are positive,
// so their bit patterns order like the values).
__global__ void anchor_argmax_kernel(const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_count,
                                     uint64_t cap, const float *__restrict__ S, const float *__restrict__ anchors,
                                     unsigned long long *__restrict__ best)
{
    uint64_t n = *cand_count;
    if (n > cap) n = cap;
    const int lane = threadIdx.x & 31;
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t k = w; k < n; k += nw) {
        const uint2 c = cand[k];
        const float2 x = __ldg(reinterpret_cast<const float2 *>(S + (int64_t)c.x * SK) + lane);
        const float2 y = __ldg(reinterpret_cast<const float2 *>(anchors + (int64_t)c.y * SK) + lane);
        float dot = fmaf(x.x, y.x, x.y * y.y);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0 && dot > 0.f)
            atomicMax(best + c.x, ((unsigned long long)__float_as_uint(dot) << 32) | (unsigned long long)c.y);
    }
}

// key[r] = anchor of best[r], or n_anchor (the group of rows no anchor reached) when best[r] == 0.
__global__ void anchor_keys_kernel(const unsigned long long *__restrict__ best, int64_t n, int n_anchor,
                                   uint32_t *__restrict__ key)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = best[r];
        key[r] = b ? (uint32_t)(b & 0xffffffffull) : (uint32_t)n_anchor;
    }
}

cudaError_t launch_anchor_argmax(const uint2 *cand, const unsigned long long *cand_count, uint64_t cap, const float *S,
                                 const float *anchors, unsigned long long *best, int num_sms, cudaStream_t st)
{
    if (cap == 0) return cudaSuccess;
    anchor_argmax_kernel<<<(unsigned)num_sms * 8, 256, 0, st>>>(cand, cand_count, cap, S, anchors, best);
    return cudaGetLastError();
}

cudaError_t launch_anchor_keys(const unsigned long long *best, int64_t n, int n_anchor, uint32_t *key, int num_sms,
                               cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 16);
    anchor_keys_kernel<<<(unsigned)blocks, 256, 0, st>>>(best, n, n_anchor, key);
    return cudaGetLastError();
}

}  // namespace ej
