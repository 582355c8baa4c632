// Tensor-core similarity contraction for sm_103a (tcgen05 + TMEM + TMA) with
// the threshold predicate and pair compaction fused into the epilogue.
//
// What it computes (Sec. IV-C, tensor formulation; Eq. Block Matrix Dot
// Product Decomposition): for every 128 x 256 tile of D = R S^T over the
// normalised rows, the FP32 accumulation of the K-slices, compared against
// the candidate threshold (Sec. III-B); the (row, col) positions that pass
// are appended to a candidate buffer (Sec. IV-C, mapping back through the
// partition offsets m0, n0).  D never leaves the chip (Sec. V-B: the
// "buffer" of a partition pair is a TMEM accumulator here).
//
// Structure (one persistent CTA per SM, 192 threads):
//   warp 0      TMA producer: 128-byte-swizzled K-slices of the R tile
//               (128 rows) and S tile (256 rows) into a 4-stage smem ring.
//   warp 1      TMEM owner and MMA issuer: 4 x tcgen05.mma per stage into one
//               of two 128 x 256 FP32 accumulators (512 TMEM columns).
//   warps 2..5  epilogue: tcgen05.ld 32 columns at a time, max-reduce for a
//               fast reject, ballot-free per-lane masks, warp prefix sums,
//               staging in shared memory, one global atomic per 1024
//               candidates (or fewer at the end).
// Every wait is bounded by `timeout` SM cycles; on expiry the CTA raises an
// abort flag, records ERR_TIMEOUT, drains its in-flight copies and MMAs,
// frees TMEM and exits.
#include "ejoin_internal.cuh"

namespace ej {

namespace {
constexpr int BM = 128, BN = 256;
constexpr int STAGES = 4;
constexpr int ROW_BYTES = 128;  // K bytes of one stage row = one 128-byte swizzle atom
constexpr int A_STAGE = BM * ROW_BYTES;
constexpr int B_STAGE = BN * ROW_BYTES;
constexpr int STAGING = 1024;  // candidate slots per epilogue warp
constexpr int EPI_WARPS = 4;
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr uint32_t TMEM_COLS = 512;
constexpr int GROUP_M = 16;

constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + STAGES * A_STAGE;
constexpr int OFF_STG = OFF_B + STAGES * B_STAGE;
constexpr int OFF_BAR = OFF_STG + EPI_WARPS * STAGING * 8;
constexpr int N_BARS = 2 * STAGES + 2 + 2 + 1;
constexpr int OFF_MISC = OFF_BAR + N_BARS * 8;
constexpr int SMEM_USED = OFF_MISC + 16;
constexpr int SMEM_BYTES = SMEM_USED + 1024;  // slack for 1024-byte alignment of the ring
static_assert(SMEM_BYTES <= 232448, "shared memory budget");

template <int KIND>
struct Kind;
template <>
struct Kind<0> {  // BF16 x BF16 -> FP32
    static constexpr int ELEMS = 64;
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(BM >> 4) << 24);
};
template <>
struct Kind<1> {  // e4m3 x e4m3 -> FP32
    static constexpr int ELEMS = 128;
    static constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(BM >> 4) << 24);
};
template <>
struct Kind<2> {  // TF32 x TF32 -> FP32
    static constexpr int ELEMS = 32;
    static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(BM >> 4) << 24);
};

template <int KIND>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum)
{
    constexpr uint32_t idesc = Kind<KIND>::IDESC;
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    } else if constexpr (KIND == 1) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    }
}

// Tile t -> (m, n): groups of GROUP_M row tiles sweep all column tiles, so the
// CTAs running concurrently share operand tiles in L2.
__device__ __forceinline__ void tile_coords(long long t, long long tiles_m, long long tiles_n, long long &m,
                                            long long &n)
{
    const long long per_group = (long long)GROUP_M * tiles_n;
    const long long g = t / per_group;
    const long long first = g * GROUP_M;
    long long gsz = tiles_m - first;
    if (gsz > GROUP_M) gsz = GROUP_M;
    const long long u = t - g * per_group;
    m = first + u % gsz;
    n = u / gsz;
}

// Wait without the abort shortcut (used only to drain in-flight work at exit).
__device__ __forceinline__ void mbar_drain_wait(uint32_t bar, uint32_t parity, uint64_t timeout, unsigned *status)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if ((uint64_t)(clock64() - t0) > timeout) {
            atomicOr(status, ERR_TIMEOUT);
            return;
        }
    }
}
}  // namespace

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
    sim_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int kp,
                  const long long *__restrict__ nA_ptr, const long long *__restrict__ nB_ptr, float thr,
                  const float *__restrict__ scaleA, const float *__restrict__ scaleB, uint2 *__restrict__ cand,
                  uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout, int count_only)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + OFF_BAR;
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
    const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(smem + OFF_MISC);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + OFF_MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long nA = *nA_ptr, nB = *nB_ptr;
    const long long tiles_m = (nA + BM - 1) / BM, tiles_n = (nB + BN - 1) / BN;
    const long long total = tiles_m * tiles_n;
    const int num_kb = kp / Kind<KIND>::ELEMS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), EPI_WARPS);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_holder), TMEM_COLS);
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
                long long m, n;
                tile_coords(t, tiles_m, tiles_n, m, n);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, timeout, abort_flag, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(full_bar(stage), A_STAGE + B_STAGE);
                    tma_load_2d(sbase + OFF_A + stage * A_STAGE, &tmA, full_bar(stage), kb * Kind<KIND>::ELEMS,
                                (int)(m * BM));
                    tma_load_2d(sbase + OFF_B + stage * B_STAGE, &tmB, full_bar(stage), kb * Kind<KIND>::ELEMS,
                                (int)(n * BN));
                    ++issued;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            // drain: every issued copy must have landed before the CTA exits
            for (int s = 0; s < STAGES; ++s) {
                if ((uint64_t)s < issued) {
                    const uint64_t last = (uint64_t)s + (uint64_t)STAGES * ((issued - 1 - (uint64_t)s) / STAGES);
                    mbar_drain_wait(full_bar(s), (uint32_t)((last / STAGES) & 1u), timeout, status);
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
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait_bounded(full_bar(stage), phase, timeout, abort_flag, status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = sbase + OFF_A + stage * A_STAGE;
                    const uint32_t b0 = sbase + OFF_B + stage * B_STAGE;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        umma<KIND>(d_tmem, sw128_kmajor_desc(a0 + 32u * k), sw128_kmajor_desc(b0 + 32u * k),
                                   (kb | k) != 0 ? 1u : 0u);
                    }
                    tc_commit(empty_bar(stage));
                    if (++stage == STAGES) {
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
            // drain: all issued MMAs complete before TMEM is released
            tc_commit(drain_bar);
            mbar_drain_wait(drain_bar, 0u, timeout, status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - 2;
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        uint2 *stg = reinterpret_cast<uint2 *>(smem + OFF_STG) + e * STAGING;
        int stg_cnt = 0;
        unsigned long long counted = 0;
        int acc = 0;
        uint32_t acc_phase = 0;

        auto flush = [&]() {
            __syncwarp();
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(cand_count, (unsigned long long)stg_cnt);
            base = __shfl_sync(0xffffffffu, base, 0);
            for (int x = lane; x < stg_cnt; x += 32) {
                const unsigned long long p = base + (unsigned long long)x;
                if (p < cap) cand[p] = stg[x];
            }
            __syncwarp();
            stg_cnt = 0;
        };

        for (long long t = blockIdx.x; t < total; t += gridDim.x) {
            long long m, n;
            tile_coords(t, tiles_m, tiles_n, m, n);
            int ok = 0;
            if (lane == 0) ok = mbar_wait_bounded(tfull_bar(acc), acc_phase, timeout, abort_flag, status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();

            const long long row = m * BM + q * 32 + lane;
            const bool row_ok = row < nA;
            float rs = 1.f;
            if (KIND == 1) rs = row_ok ? scaleA[row] : 0.f;
            const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);

#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                const long long col0 = n * BN + c * 32;
                uint32_t v[32];
                tmem_ld_32cols(tbase + (uint32_t)(c * 32), v);
                float csc = 1.f;
                if (KIND == 1) {
                    const long long cl = col0 + lane;
                    csc = cl < nB ? scaleB[cl] : 0.f;
                }
                tmem_wait_ld();
                float f[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    f[k] = __uint_as_float(v[k]);
                    if (KIND == 1) f[k] *= rs * __shfl_sync(0xffffffffu, csc, k);
                }
                float mx = f[0];
#pragma unroll
                for (int k = 1; k < 32; ++k) mx = fmaxf(mx, f[k]);
                const bool hit = row_ok && (mx >= thr);
                if (__any_sync(0xffffffffu, hit)) {
                    unsigned mask = 0u;
                    if (row_ok) {
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            if (f[k] >= thr && col0 + k < nB) mask |= 1u << k;
                    }
                    const int cnt = __popc(mask);
                    int incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int tot = __shfl_sync(0xffffffffu, incl, 31);
                    if (count_only) {
                        counted += (unsigned long long)tot;
                    } else if (tot) {
                        if (stg_cnt + tot > STAGING) flush();
                        int pos = stg_cnt + incl - cnt;
                        while (mask) {
                            const int k = __ffs(mask) - 1;
                            mask &= mask - 1u;
                            stg[pos++] = make_uint2((uint32_t)row, (uint32_t)(col0 + k));
                        }
                        stg_cnt += tot;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(acc));
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
        }
        if (stg_cnt) flush();
        if (count_only && lane == 0 && counted) atomicAdd(cand_count, counted);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

size_t sim_tc_smem_bytes() { return (size_t)SMEM_BYTES; }

cudaError_t launch_sim_tc(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                          const long long *nB, float thr, const float *scaleA, const float *scaleB, uint2 *cand,
                          uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout,
                          int count_only, int grid, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    switch (kind) {
    case 0:
        e = cudaFuncSetAttribute(sim_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        sim_tc_kernel<0><<<grid, THREADS, SMEM_BYTES, st>>>(*tmA, *tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap,
                                                            cand_count, status, timeout, count_only);
        break;
    case 1:
        e = cudaFuncSetAttribute(sim_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        sim_tc_kernel<1><<<grid, THREADS, SMEM_BYTES, st>>>(*tmA, *tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap,
                                                            cand_count, status, timeout, count_only);
        break;
    case 2:
        e = cudaFuncSetAttribute(sim_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        sim_tc_kernel<2><<<grid, THREADS, SMEM_BYTES, st>>>(*tmA, *tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap,
                                                            cand_count, status, timeout, count_only);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ej
