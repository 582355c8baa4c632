// ℰ-selection over a batch of query vectors (Sec. III-C, Eq. (ℰ-Selection): σ_θ over ℰ_μ(R) with
// θ a cosine predicate against each query; its cost |R|·(A + M + C), Sec. IV-A, is one scan of R).
// For every row r of R and query q of the batch, r is kept for q when cos(r, q) >= eps.
//
// The scan is HBM-bound: each row of R is read once, as raw FP32, straight from the caller's matrix.
// One persistent CTA per SM:
//   warp 0      TMA producer: 128-byte K-slices of 128 rows of R and of the (normalised, FP32) queries
//               into an 8-stage shared-memory ring.
//   warp 1      MMA issuer: tcgen05.mma kind::tf32, M = 128 rows, N = 64 queries, into one of two
//               TMEM accumulators (128 columns).
//   warps 2..5  row norms: each lane reads its row's 32 floats of every stage from shared memory and
//               accumulates the sum of squares (per-stage partial sums, compensated across stages),
//               so that the row never has to be read a second time for its norm.
//   warps 6..9  epilogue: the candidate test acc >= (eps - band) * ||r|| (q normalised: acc / ||r||
//               is the TF32 cosine, within band of the exact one), the row's 1/||r|| for the re-score,
//               and compaction of (row, col_base + query) candidates.
// The exact decision is made afterwards by the threshold join's re-score from the FP32 rows.
// Rows whose sum of squares overflows or underflows FP32 are flagged (ERR_RANGE) and the host runs
// the batch again through the normalisation pass, which rescales such rows.
#include "ejoin_internal.cuh"

namespace ej {

namespace {

constexpr int EB_M = 128, EB_N = 64;
constexpr int E_STAGES = 8;
constexpr int E_A_STAGE = EB_M * 128;
constexpr int E_B_STAGE = EB_N * 128;
constexpr int E_THREADS = 10 * 32;
constexpr uint32_t E_TMEM_COLS = 2 * EB_N;
constexpr uint32_t E_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(EB_N >> 3) << 17) |
                             ((uint32_t)(EB_M >> 4) << 24);  // TF32 x TF32 -> FP32, K-major A and B

constexpr int E_OFF_A = 0;
constexpr int E_OFF_B = E_OFF_A + E_STAGES * E_A_STAGE;
constexpr int E_OFF_NORM = E_OFF_B + E_STAGES * E_B_STAGE;  // [2][128] sums of squares
constexpr int E_OFF_BAR = E_OFF_NORM + 2 * EB_M * 4;
constexpr int E_N_BARS = 2 * E_STAGES + 6 + 1;
constexpr int E_OFF_MISC = E_OFF_BAR + E_N_BARS * 8;
constexpr int E_SMEM_BYTES = E_OFF_MISC + 16 + 1024;
static_assert(E_SMEM_BYTES <= 232448, "shared memory budget");

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(E_IDESC), "r"(accum));
}


__global__ void __launch_bounds__(E_THREADS, 1)
    esel_kernel(const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmQ, int num_kb,
                const long long *__restrict__ nR_ptr, int m, int col_base, float thr_rel,
                float *__restrict__ inv_out,
                uint2 *__restrict__ cand, uint64_t cap, unsigned long long *cand_count, unsigned *status,
                uint64_t timeout)
{
    extern __shared__ uint8_t esmem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(esmem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + E_OFF_BAR;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (E_STAGES + s); };
    auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * E_STAGES + b); };
    auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * E_STAGES + 2 + b); };
    auto nfull_bar = [&](int b) { return bar0 + 8u * (2 * E_STAGES + 4 + b); };
    const uint32_t drain_bar = bar0 + 8u * (2 * E_STAGES + 6);
    float *norm_s = reinterpret_cast<float *>(smem + E_OFF_NORM);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + E_OFF_MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + E_OFF_MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long nR = *nR_ptr;
    const long long total = (nR + EB_M - 1) / EB_M;

    if (threadIdx.x == 0) {
        for (int s = 0; s < E_STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1 + 4);  // the MMA commit and the four norm warps
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), 4);
            mbar_init(nfull_bar(b), 4);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmR);
        tma_prefetch_desc(&tmQ);
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_holder), E_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint64_t issued = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, timeout, abort_flag, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(full_bar(stage), E_A_STAGE + E_B_STAGE);
                    tma_load_2d(sbase + E_OFF_A + stage * E_A_STAGE, &tmR, full_bar(stage), kb * 32,
                                (int)(t * EB_M));
                    tma_load_2d(sbase + E_OFF_B + stage * E_B_STAGE, &tmQ, full_bar(stage), kb * 32, 0);
                    ++issued;
                    if (++stage == E_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            for (int s = 0; s < E_STAGES; ++s) {
                if ((uint64_t)s < issued) {
                    const uint64_t last = (uint64_t)s + (uint64_t)E_STAGES * ((issued - 1 - (uint64_t)s) / E_STAGES);
                    mbar_drain_wait(full_bar(s), (uint32_t)((last / E_STAGES) & 1u), status);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                if (!mbar_wait_bounded(tempty_bar(acc), acc_phase ^ 1u, timeout, abort_flag, status)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * EB_N);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait_bounded(full_bar(stage), phase, timeout, abort_flag, status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = sbase + E_OFF_A + stage * E_A_STAGE;
                    const uint32_t b0 = sbase + E_OFF_B + stage * E_B_STAGE;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        umma_tf32(d_tmem, sw128_kmajor_desc(a0 + 32u * k), sw128_kmajor_desc(b0 + 32u * k),
                                  (kb | k) != 0 ? 1u : 0u);
                    tc_commit(empty_bar(stage));
                    if (++stage == E_STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                tc_commit(tfull_bar(acc));
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1u;
                }
            }
            tc_commit(drain_bar);
            mbar_drain_wait(drain_bar, 0u, status);
        }
        __syncwarp();
    } else if (warp < 6) {
        // ------------------------------------------------------------ row norms
        const int nw = warp - 2;
        const int r = nw * 32 + lane;  // row of the tile
        int stage = 0;
        uint32_t phase = 0;
        int acc = 0;
        uint32_t acc_phase = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
            float s = 0.f, c = 0.f, mx = 0.f;  // running sum of squares, its compensation, max |x|
            bool nan_seen = false;             // a NaN element (fmaxf passes NaN over, the sums do not)
            for (int kb = 0; kb < num_kb; ++kb) {
                // every lane waits: each reads the bytes the TMA wrote
                const bool w = mbar_wait_bounded(full_bar(stage), phase, timeout, abort_flag, status);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
                // the row's 128 bytes of this stage, 16-byte chunk j ^ (lane & 7) at step j: the rows of a
                // quarter-warp start on the same bank, so this order puts their chunks on distinct banks
                // (and the sum of squares does not depend on the order)
                const float4 *row = reinterpret_cast<const float4 *>(smem + E_OFF_A + stage * E_A_STAGE + r * 128);
                float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 v = row[j ^ (lane & 7)];
                    p0 = fmaf(v.x, v.x, p0);
                    p1 = fmaf(v.y, v.y, p1);
                    p2 = fmaf(v.z, v.z, p2);
                    p3 = fmaf(v.w, v.w, p3);
                    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
                }
                const float part = (p0 + p1) + (p2 + p3);
                nan_seen |= part != part;
                // compensated accumulation across stages (Kahan)
                const float y = part - c;
                const float tt = s + y;
                c = (tt - s) - y;
                s = tt;
                __syncwarp();
                if (lane == 0) mbar_arrive(empty_bar(stage));
                if (++stage == E_STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
            // every lane waits until the epilogue has read this buffer's sums of the previous tile
            const bool w = mbar_wait_bounded(tempty_bar(acc), acc_phase ^ 1u, timeout, abort_flag, status);
            if (!__all_sync(0xffffffffu, w)) break;
            const long long row_g = t * EB_M + r;
            // NaN or Inf elements: non-finite input.  A finite row whose sum of squares overflowed (the
            // compensation then turns Inf into NaN) or underflowed: out of range, rescaled by the host's
            // second pass
            if (row_g < nR) {
                if (nan_seen || isinf(mx)) atomicOr(status, ERR_NONFINITE);
                else if (!isfinite(s) || (mx > 0.f && s < 0x1p-96f)) atomicOr(status, ERR_RANGE);
            }
            norm_s[acc * EB_M + r] = s;
            __syncwarp();
            if (lane == 0) mbar_arrive(nfull_bar(acc));
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;  // TMEM lane quarter of this warp
        const int r = q * 32 + lane;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (long long t = blockIdx.x; t < total; t += gridDim.x) {
            // every lane waits for the sums of squares it reads; the accumulator wait is lane 0's
            int w = 0;
            if (lane == 0) w = mbar_wait_bounded(tfull_bar(acc), acc_phase, timeout, abort_flag, status) ? 1 : 0;
            w = __shfl_sync(0xffffffffu, w, 0);
            const bool wn = w && mbar_wait_bounded(nfull_bar(acc), acc_phase, timeout, abort_flag, status);
            if (!__all_sync(0xffffffffu, wn)) break;
            tc_fence_after();
            const long long row = t * EB_M + r;
            const bool row_ok = row < nR;
            const float nr = sqrtf(norm_s[acc * EB_M + r]);
            const float thr_raw = thr_rel * nr;
            if (inv_out && row_ok) inv_out[row] = nr > 0.f ? 1.f / nr : 0.f;
#pragma unroll
            for (int ch = 0; ch < EB_N / 32; ++ch) {
                uint32_t v[32];
                tmem_ld_32cols(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * EB_N + ch * 32), v);
                tmem_wait_ld_regs(v);
                unsigned mask = 0u;
#pragma unroll
                for (int k = 0; k < 32; ++k) mask |= (__uint_as_float(v[k]) >= thr_raw ? 1u : 0u) << k;
                const int left = m - ch * 32;  // valid query columns in this chunk
                if (left < 32) mask &= left <= 0 ? 0u : ((1u << left) - 1u);
                if (!row_ok) mask = 0u;
                const int cnt = __popc(mask);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                if (tot) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(cand_count, (unsigned long long)tot);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    unsigned long long p = base + (unsigned long long)(incl - cnt);
                    while (mask) {
                        const int k = __ffs(mask) - 1;
                        mask &= mask - 1u;
                        if (p < cap) cand[p] = make_uint2((uint32_t)row, (uint32_t)(col_base + ch * 32 + k));
                        ++p;
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(acc));
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, E_TMEM_COLS);
}

}  // namespace

cudaError_t launch_esel(const CUtensorMap *tmR, const CUtensorMap *tmQ, int num_kb, const long long *nR, int m,
                        int col_base, float thr_rel, float *inv_out, uint2 *cand, uint64_t cap,
                        unsigned long long *cand_count, unsigned *status, uint64_t timeout, int grid, cudaStream_t st)
{
    if (m < 1 || m > EB_N || num_kb < 1) return cudaErrorInvalidValue;
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!((configured >> dev) & 1ull)) {
        e = cudaFuncSetAttribute(esel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured |= 1ull << dev;
    }
    esel_kernel<<<grid, E_THREADS, E_SMEM_BYTES, st>>>(*tmR, *tmQ, num_kb, nR, m, col_base, thr_rel, inv_out, cand,
                                                       cap, cand_count, status, timeout);
    return cudaGetLastError();
}

}  // namespace ej
