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
// Structure (one persistent CTA per SM, 320 threads; 576 for e4m3 at short K):
//   warp 0      TMA producer: 128-byte-swizzled K-slices of the R tile
//               (128 rows) and S tile (256 rows) into a 4-stage smem ring.
//   warp 1      TMEM owner and MMA issuer: 4 x tcgen05.mma per stage into one
//               of two 128 x 256 FP32 accumulators (512 TMEM columns).
//   warps 2..    epilogue, two (e4m3 at short K: four) warps per TMEM lane
//               quarter, each on 128 (64) of the 256 accumulator columns:
//               software-pipelined tcgen05.ld of 32 columns, tree
//               max-reduce for a fast reject, per-lane match
//               masks, warp prefix sums, staging in shared memory, one global
//               atomic per flush of up to 512 candidates.
// Every wait is bounded by `timeout` SM cycles; on expiry the CTA raises an
// abort flag, records ERR_TIMEOUT, drains its in-flight copies and MMAs (with
// a fixed bound of its own, not `timeout`: issued work always completes),
// frees TMEM and exits.
#include "ejoin_internal.cuh"

namespace ej {

namespace {
constexpr int BM = 128, BN = 256;
constexpr int STAGES = 4;
constexpr int ROW_BYTES = 128;  // K bytes of one stage row = one 128-byte swizzle atom
constexpr int A_STAGE = BM * ROW_BYTES;
constexpr int B_STAGE = BN * ROW_BYTES;
constexpr int FLUSH_TILES = 16;  // tiles between candidate flushes of an epilogue warp (or when staging is full)
// Epilogue warps: the same number per TMEM lane quarter, each on a slice of the accumulator columns.  An
// e4m3 tile of short K (at most 512 values, 4 K-slices) takes too little MMA time for 8 warps to scan its
// accumulator, so its epilogue is split over 16 warps (64 columns each); longer K and BF16 / TF32 use 8
// (128 columns each), which leaves the MMA warp's scheduler less crowded.
constexpr int EPI_WIDE_MAX_KP = 512;
constexpr int epi_warps(int kind, bool wide) { return kind == 1 && wide ? 16 : 8; }
constexpr int EPI_WARPS_MAX = 16;
constexpr int STAGING_BYTES = 32768;  // candidate staging of all epilogue warps
// fused re-score: the warps after the epilogue warps consume candidates from a shared-memory ring that
// replaces the epilogue staging: QN cells of 8 data bytes, QN 32-bit cell sequence numbers,
// then RS_STG staged result records per re-score warp
constexpr int RS_WARPS_F = 4;
constexpr int QN = 2048;
constexpr int RS_STG = 128;
constexpr uint32_t TMEM_COLS = 512;

constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + STAGES * A_STAGE;
constexpr int OFF_STG = OFF_B + STAGES * B_STAGE;
constexpr int OFF_CTR = OFF_STG + STAGING_BYTES;
constexpr int OFF_BAR = OFF_CTR + EPI_WARPS_MAX * 4;
static_assert(QN * 12 + RS_WARPS_F * RS_STG * 12 <= STAGING_BYTES, "fused ring fits the staging area");
static_assert(EPI_WARPS_MAX * 4 >= 12, "fused ring counters");
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

// Tile t -> (m, n): groups of group_m row tiles sweep all column tiles, so the
// CTAs running concurrently share operand tiles in L2, and the candidates they
// emit (which the re-score gathers in emission order) touch a bounded set of
// FP32 input rows.
__device__ __forceinline__ void tile_coords(long long t, long long tiles_m, long long tiles_n, int group_m,
                                            long long &m, long long &n)
{
    if (tiles_m * tiles_n < 0x7fffffffll && (long long)group_m * tiles_n < 0x7fffffffll) {
        // 32-bit arithmetic (a 64-bit division is a long software sequence, paid per tile by every role)
        const uint32_t tt = (uint32_t)t, tm = (uint32_t)tiles_m;
        const uint32_t per_group = (uint32_t)group_m * (uint32_t)tiles_n;
        const uint32_t g = tt / per_group;
        const uint32_t first = g * (uint32_t)group_m;
        const uint32_t gsz = min(tm - first, (uint32_t)group_m);
        const uint32_t u = tt - g * per_group;
        const uint32_t nn = u / gsz;
        m = first + (u - nn * gsz);
        n = nn;
        return;
    }
    const long long per_group = (long long)group_m * tiles_n;
    const long long g = t / per_group;
    const long long first = g * group_m;
    long long gsz = tiles_m - first;
    if (gsz > group_m) gsz = group_m;
    const long long u = t - g * per_group;
    m = first + u % gsz;
    n = u / gsz;
}

// Where a tile of the global tile space lives: first operand rows of R and S,
// valid extents inside the tile, threshold.
struct TileInfo {
    long long rowA, rowB;
    int limA, limB;
    float thr;
    bool diag;  // MODE_SYM: a tile of a diagonal block (keep col >= row only)
};

enum : int { MODE_SINGLE = 0, MODE_BATCH = 1, MODE_LIST = 2, MODE_FUSED = 3, MODE_SYM = 4, MODE_TOPMAX = 5,
             MODE_TOPCAND = 6, MODE_TOP1 = 7, MODE_GEMM = 8 };
// MODE_GEMM: the accumulator tile is written out as a dense layer (row scale, bias, activation) instead
// of being compared with a threshold: the sketch network's layers on the tensor cores.
// MODE_TOPMAX / MODE_TOPCAND: the two contraction passes of the top-k join condition (Sec. VI-E),
// tiled like MODE_SINGLE.  TOPMAX keeps, per row of A and column group, the largest bulk similarity
// over the valid columns (no candidates); TOPCAND emits the candidates within a margin of a per-row
// threshold.  MODE_TOP1: top-1 in one pass.  Each lane emits a 32-column chunk's columns within the
// margin of its row's running maximum (read at the tile start) merged with the row's maximum over
// the tile's chunks so far, this chunk included, and raises the running maximum at the tile end
// (atomicMax).  Every such threshold is at most the final row maximum less the margin, so the
// column of the exact maximum, within the margin of the final one, is always emitted.

// MODE_SYM (self-join, R == S): only the block pairs (I, J), I <= J, of
// 256-row blocks are contracted, each as its two 128-row tiles (2I, J) and
// (2I + 1, J); inside a diagonal block (I == J) only the positions with
// col >= row are kept.  Every unordered pair is found once and the re-score
// emits it in both orders.  Raster: groups of G block rows; inside a group,
// column blocks J = I0 .. nb - 1 in order, and for each J the group's block
// rows I0 .. min(I0 + G, J + 1) - 1.
struct SymRaster {
    long long nb;  // 256-row blocks
    long long G;   // block rows per group
};

// Tiles (two per block pair) of the full groups 0 .. g - 1 (each with nb - I0 >= G columns).
__device__ __forceinline__ long long sym_group_start(long long g, const SymRaster &sr)
{
    const long long G = sr.G;
    return g * G * (G + 1) + 2 * G * (g * (sr.nb - G) - G * (g * (g - 1) / 2));
}

__device__ __forceinline__ long long sym_total(const SymRaster &sr) { return sr.nb * (sr.nb + 1); }

// Tile t of the symmetric raster -> (m, n, diagonal block?)
__device__ __forceinline__ void sym_coords(long long t, const SymRaster &sr, long long &m, long long &n, bool &diag)
{
    const long long G = sr.G;
    const long long n_groups = (sr.nb + G - 1) / G;
    // group: the last g with start(g) <= t (starts of the full groups grow with g)
    long long lo = 0, hi = n_groups;  // start(lo) <= t < start(hi) (start(n_groups) taken as +inf)
    while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        if (sym_group_start(mid, sr) <= t) lo = mid;
        else hi = mid;
    }
    const long long I0 = lo * G;
    const long long Gg = min(G, sr.nb - I0);
    const long long u = t - sym_group_start(lo, sr);
    const long long b = u >> 1;  // block pair inside the group
    const long long h = u & 1;   // which 128-row half of the block row
    const long long L = sr.nb - I0;
    const long long tri_cols = min(L, Gg);
    const long long tri = tri_cols * (tri_cols + 1) / 2;
    long long x, y;
    if (b < tri) {
        // column x holds x + 1 block rows: largest x with x (x + 1) / 2 <= b (b < G (G + 1) / 2 is small:
        // the single-precision root is within one of x, and the loops below correct it)
        x = (long long)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
        while (x * (x + 1) / 2 > b) --x;
        while ((x + 1) * (x + 2) / 2 <= b) ++x;
        y = b - x * (x + 1) / 2;
    } else {
        const long long r = b - tri;
        x = tri_cols + r / Gg;
        y = r % Gg;
    }
    m = 2 * (I0 + y) + h;
    n = I0 + x;
    diag = x == y;
}

constexpr int threads_for(int ew, int mode) { return (2 + ew + (mode == MODE_FUSED ? RS_WARPS_F : 0)) * 32; }

// Re-score role of the fused kernel: take 8 queue slots at a time, gather the
// FP32 rows of up to 8 candidates at once, FP32 dot (FP64 tier inside the
// band), emit pairs with sim >= eps through a staged, one-atomic-per-flush
// output.  Exits when every epilogue warp is done and the queue is drained.
__device__ __forceinline__ void rescore_role(uint8_t *smem, const FuseArgs &fa, volatile int *abort_flag,
                                             unsigned *status, uint64_t timeout, int rw, int lane,
                                             unsigned long long *band_count_total, int n_epi)
{
    // bounded multi-producer / multi-consumer ring with per-cell sequence numbers: the producer
    // of position p waits for seq == p, writes, sets seq = p + 1; the consumer of p waits for
    // seq == p + 1, reads, sets seq = p + QN (the cell is free for position p + QN)
    volatile unsigned long long *vq = reinterpret_cast<volatile unsigned long long *>(smem + OFF_STG);
    volatile uint32_t *vseq = reinterpret_cast<volatile uint32_t *>(smem + OFF_STG + QN * 8);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(smem + OFF_CTR);  // [0] head, [1] take, [2] producers done
    volatile uint32_t *vctr = ctr;
    uint32_t *stg = reinterpret_cast<uint32_t *>(smem + OFF_STG + QN * 12) + rw * RS_STG * 3;
    int stg_n = 0;
    unsigned long long n_band = 0;
    const int d4 = fa.d >> 2;
    uint32_t *out_w = reinterpret_cast<uint32_t *>(fa.out);

    auto flush = [&]() {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0 && stg_n) base = atomicAdd(fa.pair_count, (unsigned long long)stg_n);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (!fa.count_only) {
            for (int x = lane; x < 3 * stg_n; x += 32)
                if (base + (unsigned long long)(x / 3) < fa.out_cap) out_w[base * 3 + x] = stg[x];
        }
        __syncwarp();
        stg_n = 0;
    };

    while (true) {
        uint32_t s0 = 0;
        if (lane == 0) s0 = atomicAdd(&ctr[1], 8u);
        s0 = __shfl_sync(0xffffffffu, s0, 0);
        uint32_t row = 0, col = 0;
        bool valid = false, ended = false;
        if (lane < 8) {
            const uint32_t sl = s0 + (uint32_t)lane;
            const int slot = (int)(sl & (QN - 1));
            const long long t0 = clock64();
            while (true) {
                if (vseq[slot] == sl + 1u) {
                    __threadfence_block();
                    const unsigned long long e = vq[slot];
                    row = (uint32_t)e;
                    col = (uint32_t)(e >> 32);
                    __threadfence_block();
                    vseq[slot] = sl + (uint32_t)QN;  // the cell is free for position sl + QN
                    valid = true;
                    break;
                }
                if (vctr[2] == (uint32_t)n_epi && sl >= vctr[0]) {
                    ended = true;  // every candidate has been queued, and none at this position
                    break;
                }
                if (*abort_flag) {
                    ended = true;
                    break;
                }
                if ((uint64_t)(clock64() - t0) > timeout) {
                    *abort_flag = 1;
                    atomicOr(status, ERR_TIMEOUT);
                    ended = true;
                    break;
                }
            }
        }
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        const bool any_end = __any_sync(0xffffffffu, ended);
        if (vm) {
            const float4 *pr[8], *ps[8];
            uint32_t gi[8], gj[8];
            float sc[8], acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint32_t ri = __shfl_sync(0xffffffffu, row, c), cj = __shfl_sync(0xffffffffu, col, c);
                const bool v = (vm >> c) & 1u;
                gi[c] = v ? (fa.idsR ? fa.idsR[ri] : ri) : 0u;
                gj[c] = v ? (fa.idsS ? fa.idsS[cj] : cj) : 0u;
                sc[c] = v ? fa.invR[ri] * fa.invS[cj] : 0.f;
                pr[c] = reinterpret_cast<const float4 *>(fa.R + (int64_t)gi[c] * fa.ldR);
                ps[c] = reinterpret_cast<const float4 *>(fa.S + (int64_t)gj[c] * fa.ldS);
                acc[c] = 0.f;
            }
            for (int g = lane; g < d4; g += 32) {
                float4 a[8], b[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const bool v = (vm >> c) & 1u;
                    a[c] = v ? __ldg(pr[c] + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                    b[c] = v ? __ldg(ps[c] + g) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    acc[c] = fmaf(a[c].x, b[c].x, acc[c]);
                    acc[c] = fmaf(a[c].y, b[c].y, acc[c]);
                    acc[c] = fmaf(a[c].z, b[c].z, acc[c]);
                    acc[c] = fmaf(a[c].w, b[c].w, acc[c]);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
            bool my_emit = false;
            uint32_t my_i = 0, my_j = 0;
            float my_sim = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (!((vm >> c) & 1u)) continue;  // warp-uniform
                float sim = fminf(1.f, fmaxf(-1.f, acc[c] * sc[c]));
                bool emit = sim >= fa.eps;
                if (fabsf(sim - fa.eps) < fa.fp64_band) {
                    // accurate tier: compensated dot product and norms, finished in FP64
                    const double s64 = accurate_cosine(fa.R + (int64_t)gi[c] * fa.ldR, fa.S + (int64_t)gj[c] * fa.ldS,
                                                       fa.d, lane);
                    emit = s64 >= (double)fa.eps;
                    sim = (float)s64;
                    ++n_band;
                }
                if (lane == c) {
                    my_emit = emit;
                    my_i = gi[c];
                    my_j = gj[c];
                    my_sim = sim;
                }
            }
            const unsigned em = __ballot_sync(0xffffffffu, my_emit);
            if (em) {
                if (stg_n + __popc(em) > RS_STG) flush();
                if (my_emit) {
                    const int pos = stg_n + __popc(em & ((1u << lane) - 1u));
                    stg[3 * pos + 0] = my_i;
                    stg[3 * pos + 1] = my_j;
                    stg[3 * pos + 2] = __float_as_uint(my_sim);
                }
                stg_n += __popc(em);
                __syncwarp();
            }
        }
        if (any_end) break;
    }
    flush();
    if (lane == 0 && n_band) atomicAdd(band_count_total, n_band);
}

// max(a, b, c) in one instruction (three-input max.f32, sm_100 and later); the operands are finite
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <int MODE>
__device__ __forceinline__ TileInfo decode_tile(long long t, const BatchTables &bt, long long tiles_m,
                                                long long tiles_n, long long nA, long long nB, float thr, int group_m,
                                                long long col_stride, int &job)
{
    TileInfo ti;
    ti.diag = false;
    long long m, n;
    if constexpr (MODE == MODE_SYM) {
        const SymRaster sr{(nA + 2 * BM - 1) / (2 * BM), group_m > 2 ? (long long)(group_m / 2) : 1ll};
        sym_coords(t, sr, m, n, ti.diag);
        ti.rowA = m * BM;
        ti.rowB = n * BN;
        ti.limA = (int)max(-1ll, min((long long)BM, nA - m * BM));  // <= 0: the empty half of a last block
        ti.limB = (int)min((long long)BN, nB - n * BN);
        ti.thr = thr;
    } else if constexpr (MODE == MODE_LIST) {
        const uint2 mn = __ldg(bt.tile_list + t);
        m = mn.x;
        n = mn.y;
        ti.diag = bt.sym && (m >> 1) == n;
        ti.rowA = m * BM;
        ti.rowB = n * BN;
        ti.limA = (int)min((long long)BM, nA - m * BM);
        ti.limB = (int)min((long long)BN, nB - n * BN);
        ti.thr = thr;
    } else if constexpr (MODE == MODE_BATCH) {
        // the job holding tile t: a CTA visits its tiles in increasing order, so `job` (the previous tile's
        // job, 0 at the start) only moves forward, one job table entry at a time
        int lo = job;
        while (lo + 1 < bt.n_jobs && __ldg(bt.tile_off + lo + 1) <= t) ++lo;
        job = lo;
        const long long na = __ldg(bt.nA + lo), nb = __ldg(bt.nB + lo);
        tile_coords(t - __ldg(bt.tile_off + lo), (na + BM - 1) / BM, (nb + BN - 1) / BN, group_m, m, n);
        ti.rowA = __ldg(bt.a_off + lo) + m * BM;
        ti.rowB = __ldg(bt.b_off + lo) + n * BN;
        ti.limA = (int)min((long long)BM, na - m * BM);
        ti.limB = (int)min((long long)BN, nb - n * BN);
        ti.thr = __ldg(bt.thr + lo);
    } else {
        tile_coords(t, tiles_m, tiles_n, group_m, m, n);
        n *= col_stride;
        ti.rowA = m * BM;
        ti.rowB = n * BN;
        ti.limA = (int)min((long long)BM, nA - m * BM);
        ti.limB = (int)min((long long)BN, nB - n * BN);
        ti.thr = thr;
    }
    return ti;
}

}  // namespace

template <int KIND, int MODE, int EW>
__global__ void __launch_bounds__(threads_for(EW, MODE), 1)
    sim_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int kp,
                  const long long *__restrict__ nA_ptr, const long long *__restrict__ nB_ptr, float thr,
                  const float *__restrict__ scaleA, const float *__restrict__ scaleB, uint2 *__restrict__ cand,
                  uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout, int count_only,
                  int group_m, const BatchTables bt, const FuseArgs fa)
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

    constexpr int EPI_WARPS = EW;
    constexpr int SLICE_COLS = BN / (EPI_WARPS / 4);  // accumulator columns per epilogue warp
    constexpr int EPI_CHUNKS = SLICE_COLS / 32;       // 32-column chunks per epilogue warp
    constexpr int STAGING = STAGING_BYTES / 8 / EPI_WARPS;  // candidate slots per epilogue warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long nA = MODE == MODE_BATCH ? 0 : *nA_ptr, nB = MODE == MODE_BATCH ? 0 : *nB_ptr;
    const long long tiles_m = (nA + BM - 1) / BM;
    // MODE_TOPMAX may sample every col_stride-th column tile, keeping at least top_min_tiles of them
    long long col_stride = 1;
    if (MODE == MODE_TOPMAX && bt.top_stride > 1) {
        const long long tn = (nB + BN - 1) / BN;
        col_stride = max(1ll, min((long long)bt.top_stride, tn / max(1ll, (long long)bt.top_min_tiles)));
    }
    const long long tiles_n = ((nB + BN - 1) / BN + col_stride - 1) / col_stride;
    long long total = tiles_m * tiles_n;
    if (MODE == MODE_BATCH) total = __ldg(bt.tile_off + bt.n_jobs);
    if (MODE == MODE_SYM) total = sym_total(SymRaster{(nA + 2 * BM - 1) / (2 * BM), 1});
    if (MODE == MODE_LIST) {
        const unsigned long long c = *bt.tile_count;
        total = (long long)(c < bt.tile_cap ? c : bt.tile_cap);
    }
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
        if (MODE == MODE_FUSED) {
            uint32_t *c32 = reinterpret_cast<uint32_t *>(smem + OFF_CTR);
            c32[0] = 0u;  // head: next position to reserve
            c32[1] = 0u;  // take: next position to consume
            c32[2] = 0u;  // epilogue warps done
        }
        fence_mbar_init();
    }
    if (MODE == MODE_FUSED) {
        uint32_t *seq = reinterpret_cast<uint32_t *>(smem + OFF_STG + QN * 8);
        for (int i = threadIdx.x; i < QN; i += blockDim.x) seq[i] = (uint32_t)i;  // cell i free for position i
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
            int job_p = 0;  // MODE_BATCH: job of the last decoded tile
            bool ok = true;
            for (long long t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const TileInfo ti =
                    decode_tile<MODE>(t, bt, tiles_m, tiles_n, nA, nB, thr, group_m, col_stride, job_p);
                for (int kb = 0; kb < num_kb; ++kb) {
                    if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, timeout, abort_flag, status)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(full_bar(stage), A_STAGE + B_STAGE);
                    tma_load_2d(sbase + OFF_A + stage * A_STAGE, &tmA, full_bar(stage), kb * Kind<KIND>::ELEMS,
                                (int)ti.rowA);
                    tma_load_2d(sbase + OFF_B + stage * B_STAGE, &tmB, full_bar(stage), kb * Kind<KIND>::ELEMS,
                                (int)ti.rowB);
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
                    mbar_drain_wait(full_bar(s), (uint32_t)((last / STAGES) & 1u), status);
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
            mbar_drain_wait(drain_bar, 0u, status);
        }
        __syncwarp();
    } else if (warp >= 2 + EPI_WARPS) {
        // ------------------------------------------------- fused re-score role
        if constexpr (MODE == MODE_FUSED)
            rescore_role(smem, fa, abort_flag, status, timeout, warp - 2 - EPI_WARPS, lane, fa.band_count,
                         EPI_WARPS);
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - 2;      // 0 .. EPI_WARPS-1
        const int q = warp & 3;      // TMEM lane quarter this warp may access
        const int slice = e >> 2;    // which SLICE_COLS accumulator columns
        uint2 *stg = reinterpret_cast<uint2 *>(smem + OFF_STG) + e * STAGING;
        int *stg_ctr = reinterpret_cast<int *>(smem + OFF_CTR) + e;  // mirrors stg_cnt for slot claims
        // (in the fused mode these words hold the queue counters, set once at kernel start)
        if (MODE != MODE_FUSED && lane == 0) *stg_ctr = 0;
        __syncwarp();
        int stg_cnt = 0;
        int job_e = 0;  // MODE_BATCH: job of the last decoded tile
        int tiles_since_flush = 0;
        unsigned long long counted = 0;
        int acc = 0;
        uint32_t acc_phase = 0;

        auto flush = [&]() {
            __syncwarp();
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(cand_count, (unsigned long long)stg_cnt);
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            for (int x = lane; x < stg_cnt; x += 32) {
                const unsigned long long p = base + (unsigned long long)x;
                if (p < cap) cand[p] = stg[x];
            }
            if (lane == 0) *stg_ctr = 0;
            __syncwarp();
            stg_cnt = 0;
        };

        for (long long t = blockIdx.x; t < total; t += gridDim.x) {
            const TileInfo ti = decode_tile<MODE>(t, bt, tiles_m, tiles_n, nA, nB, thr, group_m, col_stride, job_e);
            const float thr_t = ti.thr;
            // top-k modes: the row's threshold / running maximum, loaded before the accumulator wait so
            // that its latency hides behind the MMAs
            unsigned pre_best = 0u;
            if constexpr (MODE == MODE_TOPCAND || MODE == MODE_TOP1) {
                if (q * 32 + lane < ti.limA) pre_best = __ldcg(bt.row_best + ti.rowA + q * 32 + lane);
            }
            // e4m3 with tile-shared column scales: the row's and the tile's scales, loaded before the
            // accumulator wait for the same reason
            float pre_sa = 0.f, pre_sb = 0.f;
            if constexpr (KIND == 1 && (MODE == MODE_SINGLE || MODE == MODE_SYM || MODE == MODE_TOPMAX ||
                                        MODE == MODE_TOPCAND || MODE == MODE_TOP1)) {
                if (q * 32 + lane < ti.limA) {
                    pre_sa = scaleA[ti.rowA + q * 32 + lane];
                    pre_sb = __ldg(scaleB + ti.rowB);
                }
            }
            int ok = 0;
            if (lane == 0) ok = mbar_wait_bounded(tfull_bar(acc), acc_phase, timeout, abort_flag, status) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();

            const int row_local = q * 32 + lane;
            const bool row_ok = row_local < ti.limA;
            const long long row = ti.rowA + row_local;  // emitted operand row
            const int colbase_local = slice * SLICE_COLS;
            const long long colbase = ti.rowB + colbase_local;
            const uint32_t tbase =
                tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN) + (uint32_t)(slice * SLICE_COLS);
            // e4m3: similarity = acc * s_row * s_col.  In the single and self-join modes the rows of a
            // 256-row column tile share one scale (launch_normalize_fp8_grouped), so the two scales fold
            // into a per-lane threshold on the raw accumulator; the other modes scale every element
            constexpr bool TILE_SCALE = KIND == 1 && (MODE == MODE_SINGLE || MODE == MODE_SYM ||
                                                      MODE == MODE_TOPMAX || MODE == MODE_TOPCAND ||
                                                      MODE == MODE_TOP1);
            float sc_tile = 1.f;  // s_row * s_col of the e4m3 tile (TILE_SCALE)
            float rs = 1.f;
            float thr_lane = thr_t;
            float csc[EPI_CHUNKS];
#pragma unroll
            for (int c = 0; c < EPI_CHUNKS; ++c) csc[c] = 1.f;
            float thr_base = thr_t;
            if constexpr (MODE == MODE_TOPCAND) {
                // this row's best bulk similarity (pass 0) less the margin
                thr_base = row_ok ? ord2f(pre_best) - bt.top_margin : INFINITY;
                thr_lane = thr_base;
            }
            float lane_max = -INFINITY;  // MODE_TOPMAX, MODE_TOP1 (raw accumulator units)
            // MODE_TOP1: the row's running maximum as loaded at the tile start (it only grows, so a stale
            // value is a lower bound of the final one)
            const float best0 = pre_best ? ord2f(pre_best) : -INFINITY;
            if constexpr (TILE_SCALE) {
                const float sc = row_ok ? pre_sa * pre_sb : 0.f;
                sc_tile = sc;
                thr_lane = sc > 0.f ? __fdiv_rn(thr_base, sc) : (thr_base <= 0.f ? -INFINITY : INFINITY);
            } else if constexpr (KIND == 1) {
                rs = row_ok ? scaleA[row] : 0.f;
#pragma unroll
                for (int c = 0; c < EPI_CHUNKS; ++c) {
                    const int cl = colbase_local + c * 32 + lane;
                    csc[c] = cl < ti.limB ? scaleB[ti.rowB + cl] : 0.f;
                }
            }

            auto process = [&](uint32_t (&v)[32], int c) {
                const long long col0 = colbase + c * 32;
                const int left = ti.limB - (colbase_local + c * 32);  // valid columns in this chunk
                if constexpr (MODE == MODE_GEMM) {
                    // dense layer: each lane writes its row's 32 columns of this chunk (float4 stores)
                    if (row_ok && left > 0) {
                        const float rsc = bt.g_rowscale ? __ldg(bt.g_rowscale + row) : 1.f;
                        float *o = bt.g_out + row * bt.g_ld + col0;
#pragma unroll
                        for (int k4 = 0; k4 < 8; ++k4) {
                            float y[4];
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const int k = 4 * k4 + t;
                                float x = __uint_as_float(v[k]) * rsc;
                                if (bt.g_bias && k < left) x += __ldg(bt.g_bias + col0 + k);
                                if (bt.g_act == 1) x = 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
                                y[t] = x;
                            }
                            if (4 * k4 + 3 < left) {
                                *reinterpret_cast<float4 *>(o + 4 * k4) = make_float4(y[0], y[1], y[2], y[3]);
                            } else {
#pragma unroll
                                for (int t = 0; t < 4; ++t)
                                    if (4 * k4 + t < left) o[4 * k4 + t] = y[t];
                            }
                        }
                    }
                    __syncwarp();  // reconverge before the caller's .sync.aligned tcgen05 instructions
                    return;
                }
                float f[32];
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    f[k] = __uint_as_float(v[k]);
                    if (KIND == 1 && !TILE_SCALE) f[k] *= rs * __shfl_sync(0xffffffffu, csc[c], k);
                }
                // max tree of three-input maxima: a8[g] = max of f[8g .. 8g+7]
                float a8[4];
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const float* h = f + 8 * g;
                    a8[g] = fmax3(fmax3(h[0], h[1], h[2]), fmax3(h[3], h[4], h[5]), fmaxf(h[6], h[7]));
                }
                const float mx = fmax3(a8[0], a8[1], fmaxf(a8[2], a8[3]));
                if constexpr (MODE == MODE_TOPMAX || MODE == MODE_TOP1) {
                    // the row maximum over the valid columns only (padding columns hold zeros)
                    if (left >= 32) {
                        lane_max = fmaxf(lane_max, mx);
                    } else {
#pragma unroll
                        for (int k = 0; k < 32; ++k)
                            if (k < left) lane_max = fmaxf(lane_max, f[k]);
                    }
                }
                if constexpr (MODE == MODE_TOPMAX) return;
                if constexpr (MODE == MODE_TOP1) {
                    // threshold: the running maximum merged with this row's maximum over the chunks seen so
                    // far in this tile (this chunk included), less the margin
                    thr_lane = INFINITY;
                    if (row_ok && lane_max > -INFINITY) {
                        const float tb = fmaxf(best0, TILE_SCALE ? lane_max * sc_tile : lane_max) - bt.top_margin;
                        if constexpr (TILE_SCALE)
                            thr_lane = sc_tile > 0.f ? __fdiv_rn(tb, sc_tile) : (tb <= 0.f ? -INFINITY : INFINITY);
                        else
                            thr_lane = tb;
                    }
                }
                if (!__any_sync(0xffffffffu, row_ok && mx >= thr_lane)) return;
                // slow path: per-lane match mask, built only for 8-column groups that hold a match
                unsigned mask = 0u;
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    if (__any_sync(0xffffffffu, row_ok && a8[g] >= thr_lane)) {
#pragma unroll
                        for (int k = 0; k < 8; ++k) mask |= (f[8 * g + k] >= thr_lane ? 1u : 0u) << (8 * g + k);
                    }
                }
                if (left < 32) mask &= left <= 0 ? 0u : ((1u << left) - 1u);
                if constexpr (MODE == MODE_SYM || MODE == MODE_LIST) {
                    // diagonal block of a symmetric evaluation: keep col >= row (the mirror is emitted by
                    // the re-score)
                    if (ti.diag) {
                        const long long skip = row - col0;  // columns of this chunk left of the diagonal
                        mask &= skip <= 0 ? 0xffffffffu : (skip >= 32 ? 0u : ~((1u << skip) - 1u));
                    }
                }
                if (!row_ok) mask = 0u;
                const int cnt = __popc(mask);
                const int tot = (int)__reduce_add_sync(0xffffffffu, (unsigned)cnt);
                if constexpr (MODE == MODE_FUSED) {
                    // hand the candidates to the re-score warps through the shared-memory queue
                    counted += (unsigned long long)tot;
                    if (cnt) {
                        volatile unsigned long long *vq = reinterpret_cast<volatile unsigned long long *>(smem + OFF_STG);
                        volatile uint32_t *vseq = reinterpret_cast<volatile uint32_t *>(smem + OFF_STG + QN * 8);
                        uint32_t pos = atomicAdd(reinterpret_cast<uint32_t *>(smem + OFF_CTR), (uint32_t)cnt);
                        while (mask) {
                            const int k = __ffs(mask) - 1;
                            mask &= mask - 1u;
                            const int slot = (int)(pos & (QN - 1));
                            const long long t0 = clock64();
                            bool ok = true;
                            while (vseq[slot] != pos) {  // wait until the cell is free for this position
                                if (*abort_flag) {
                                    ok = false;
                                    break;
                                }
                                if ((uint64_t)(clock64() - t0) > timeout) {
                                    *abort_flag = 1;
                                    atomicOr(status, ERR_TIMEOUT);
                                    ok = false;
                                    break;
                                }
                            }
                            if (!ok) break;
                            vq[slot] = ((unsigned long long)(uint32_t)(col0 + k) << 32) | (uint32_t)row;
                            __threadfence_block();
                            vseq[slot] = pos + 1u;  // published
                            ++pos;
                        }
                    }
                    // reconverge: the caller's next tcgen05.wait::ld is a .sync.aligned instruction
                    __syncwarp();
                    return;
                }
                if (count_only) {
                    counted += (unsigned long long)tot;
                    return;
                }
                if (tot == 0) return;
                if (tot > STAGING) {
                    // denser than the staging area: claim space and write directly
                    int incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    unsigned long long base = 0;
                    if (lane == 0) {
                        base = atomicAdd(cand_count, (unsigned long long)tot);
                    }
                    base = __shfl_sync(0xffffffffu, base, 0);
                    unsigned long long p = base + (unsigned long long)(incl - cnt);
                    while (mask) {
                        const int k = __ffs(mask) - 1;
                        mask &= mask - 1u;
                        if (p < cap) cand[p] = make_uint2((uint32_t)row, (uint32_t)(col0 + k));
                        ++p;
                    }
                    __syncwarp();  // reconverge before the caller's .sync.aligned tcgen05 instructions
                    return;
                }
                if (stg_cnt + tot > STAGING) flush();
                if (cnt) {
                    int pos = atomicAdd(stg_ctr, cnt);  // shared-memory slot claim
                    while (mask) {
                        const int k = __ffs(mask) - 1;
                        mask &= mask - 1u;
                        stg[pos++] = make_uint2((uint32_t)row, (uint32_t)(col0 + k));
                    }
                }
                stg_cnt += tot;
                __syncwarp();
            };

            uint32_t va[32], vb[32];
            // software pipeline: the load of chunk c+1 is in flight while chunk c is scanned
            tmem_ld_32cols(tbase, va);
            tmem_wait_ld_regs(va);
#pragma unroll
            for (int c = 0; c < EPI_CHUNKS; ++c) {
                if (c + 1 < EPI_CHUNKS) {
                    if (c & 1)
                        tmem_ld_32cols(tbase + (uint32_t)((c + 1) * 32), va);
                    else
                        tmem_ld_32cols(tbase + (uint32_t)((c + 1) * 32), vb);
                }
                if (c & 1)
                    process(vb, c);
                else
                    process(va, c);
                if (c + 1 < EPI_CHUNKS) {
                    if (c & 1)
                        tmem_wait_ld_regs(va);
                    else
                        tmem_wait_ld_regs(vb);
                }
            }
            if constexpr (MODE == MODE_TOPMAX) {
                if (row_ok && lane_max > -INFINITY)
                    atomicMax(bt.row_best + row * bt.top_ld + (colbase >> bt.top_shift),
                              f2ord(TILE_SCALE ? lane_max * sc_tile : lane_max));
            }
            if constexpr (MODE == MODE_TOP1) {
                // raise the running maximum (no reply awaited)
                if (row_ok && lane_max > -INFINITY) {
                    const unsigned o = f2ord(TILE_SCALE ? lane_max * sc_tile : lane_max);
                    if (o > pre_best) atomicMax(bt.row_best + row, o);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(acc));
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1u;
            }
            // publish the staged candidates every FLUSH_TILES tiles (accumulator already released):
            // the list then follows the raster closely, and the re-score's row gathers stay in L2
            if constexpr (MODE != MODE_FUSED) {
                if (++tiles_since_flush >= FLUSH_TILES) {
                    tiles_since_flush = 0;
                    if (stg_cnt) flush();
                }
            }
        }
        if constexpr (MODE == MODE_FUSED) {
            __threadfence_block();
            __syncwarp();
            if (lane == 0) {
                if (counted) atomicAdd(cand_count, counted);
                atomicAdd(reinterpret_cast<uint32_t *>(smem + OFF_CTR + 8), 1u);  // this producer is done
            }
        } else {
            if (stg_cnt) flush();
            if (count_only && lane == 0 && counted) atomicAdd(cand_count, counted);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

size_t sim_tc_smem_bytes() { return (size_t)SMEM_BYTES; }

template <int KIND, int MODE, int EW>
static cudaError_t launch_ew(const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                             const long long *nB, float thr, const float *scaleA, const float *scaleB, uint2 *cand,
                             uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout,
                             int count_only, int grid, int group_m, const BatchTables &bt, cudaStream_t st,
                             const FuseArgs &fa)
{
    // the shared-memory opt-in is set once per device (and therefore never inside a stream capture
    // that follows a first eager launch)
    static unsigned long long configured = 0ull;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!((configured >> dev) & 1ull)) {
        e = cudaFuncSetAttribute(sim_tc_kernel<KIND, MODE, EW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured |= 1ull << dev;
    }
    sim_tc_kernel<KIND, MODE, EW><<<grid, threads_for(EW, MODE), SMEM_BYTES, st>>>(
        *tmA, *tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap, cand_count, status, timeout, count_only,
        group_m < 1 ? 1 : group_m, bt, fa);
    return cudaGetLastError();
}

template <int KIND, int MODE>
static cudaError_t launch_one(const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                              const long long *nB, float thr, const float *scaleA, const float *scaleB, uint2 *cand,
                              uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout,
                              int count_only, int grid, int group_m, const BatchTables &bt, cudaStream_t st,
                              const FuseArgs &fa = FuseArgs{})
{
    if constexpr (KIND == 1) {
        if (kp <= EPI_WIDE_MAX_KP)
            return launch_ew<KIND, MODE, epi_warps(KIND, true)>(tmA, tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap,
                                                                cand_count, status, timeout, count_only, grid,
                                                                group_m, bt, st, fa);
    }
    return launch_ew<KIND, MODE, epi_warps(KIND, false)>(tmA, tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap,
                                                         cand_count, status, timeout, count_only, grid, group_m, bt,
                                                         st, fa);
}

cudaError_t launch_sim_tc(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                          const long long *nB, float thr, const float *scaleA, const float *scaleB, uint2 *cand,
                          uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout,
                          int count_only, int grid, int group_m, cudaStream_t st)
{
    const BatchTables none{};
    switch (kind) {
    case 0:
        return launch_one<0, MODE_SINGLE>(tmA, tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap, cand_count, status,
                                          timeout, count_only, grid, group_m, none, st);
    case 1:
        return launch_one<1, MODE_SINGLE>(tmA, tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap, cand_count, status,
                                          timeout, count_only, grid, group_m, none, st);
    case 2:
        return launch_one<2, MODE_SINGLE>(tmA, tmB, kp, nA, nB, thr, scaleA, scaleB, cand, cap, cand_count, status,
                                          timeout, count_only, grid, group_m, none, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sim_tc_sym(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                              float thr, const float *scale, uint2 *cand, uint64_t cap,
                              unsigned long long *cand_count, unsigned *status, uint64_t timeout, int count_only,
                              int grid, int group_m, cudaStream_t st)
{
    const BatchTables none{};
    switch (kind) {
    case 0:
        return launch_one<0, MODE_SYM>(tmA, tmB, kp, nA, nA, thr, scale, scale, cand, cap, cand_count, status, timeout,
                                       count_only, grid, group_m, none, st);
    case 1:
        return launch_one<1, MODE_SYM>(tmA, tmB, kp, nA, nA, thr, scale, scale, cand, cap, cand_count, status, timeout,
                                       count_only, grid, group_m, none, st);
    case 2:
        return launch_one<2, MODE_SYM>(tmA, tmB, kp, nA, nA, thr, scale, scale, cand, cap, cand_count, status, timeout,
                                       count_only, grid, group_m, none, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sim_tc_top(int kind, int pass, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp,
                              const long long *nA, const long long *nB, const float *scaleA, const float *scaleB,
                              unsigned *row_best, long long top_ld, int top_shift, int top_stride, int top_min_tiles,
                              float margin, uint2 *cand, uint64_t cap, unsigned long long *cand_count,
                              unsigned *status, uint64_t timeout, int grid, int group_m, cudaStream_t st)
{
    BatchTables bt{};
    bt.row_best = row_best;
    bt.top_ld = top_ld;
    bt.top_shift = top_shift;
    bt.top_stride = top_stride;
    bt.top_min_tiles = top_min_tiles;
    bt.top_margin = margin;
#define EJ_TOP(K, M)                                                                                                  \
    launch_one<K, M>(tmA, tmB, kp, nA, nB, 0.f, scaleA, scaleB, cand, cap, cand_count, status, timeout, 0, grid,      \
                     group_m, bt, st)
    if (pass == 0) {
        switch (kind) {
        case 0: return EJ_TOP(0, MODE_TOPMAX);
        case 1: return EJ_TOP(1, MODE_TOPMAX);
        case 2: return EJ_TOP(2, MODE_TOPMAX);
        default: return cudaErrorInvalidValue;
        }
    }
    if (pass == 2) {
        switch (kind) {
        case 0: return EJ_TOP(0, MODE_TOP1);
        case 1: return EJ_TOP(1, MODE_TOP1);
        case 2: return EJ_TOP(2, MODE_TOP1);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (kind) {
    case 0: return EJ_TOP(0, MODE_TOPCAND);
    case 1: return EJ_TOP(1, MODE_TOPCAND);
    case 2: return EJ_TOP(2, MODE_TOPCAND);
    default: return cudaErrorInvalidValue;
    }
#undef EJ_TOP
}

cudaError_t launch_sim_tc_batch(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp,
                                const BatchTables &bt, const float *scaleA, const float *scaleB, uint2 *cand,
                                uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout,
                                int grid, int group_m, cudaStream_t st)
{
    switch (kind) {
    case 0:
        return launch_one<0, MODE_BATCH>(tmA, tmB, kp, nullptr, nullptr, 0.f, scaleA, scaleB, cand, cap, cand_count, status,
                                   timeout, 0, grid, group_m, bt, st);
    case 1:
        return launch_one<1, MODE_BATCH>(tmA, tmB, kp, nullptr, nullptr, 0.f, scaleA, scaleB, cand, cap, cand_count, status,
                                   timeout, 0, grid, group_m, bt, st);
    case 2:
        return launch_one<2, MODE_BATCH>(tmA, tmB, kp, nullptr, nullptr, 0.f, scaleA, scaleB, cand, cap, cand_count, status,
                                   timeout, 0, grid, group_m, bt, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sim_tc_fused(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp,
                                const long long *nA, const long long *nB, float thr, const float *scaleA,
                                const float *scaleB, const FuseArgs &fa, unsigned long long *cand_count,
                                unsigned *status, uint64_t timeout, int grid, int group_m, cudaStream_t st)
{
    const BatchTables none{};
    switch (kind) {
    case 0:
        return launch_one<0, MODE_FUSED>(tmA, tmB, kp, nA, nB, thr, scaleA, scaleB, nullptr, 0, cand_count, status,
                                         timeout, fa.count_only, grid, group_m, none, st, fa);
    case 1:
        return launch_one<1, MODE_FUSED>(tmA, tmB, kp, nA, nB, thr, scaleA, scaleB, nullptr, 0, cand_count, status,
                                         timeout, fa.count_only, grid, group_m, none, st, fa);
    case 2:
        return launch_one<2, MODE_FUSED>(tmA, tmB, kp, nA, nB, thr, scaleA, scaleB, nullptr, 0, cand_count, status,
                                         timeout, fa.count_only, grid, group_m, none, st, fa);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_gemm_tc(const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                           const long long *nB, const float *rowscale, const float *bias, int act, float *out,
                           long long out_ld, unsigned *status, uint64_t timeout, int grid, cudaStream_t st)
{
    if (out_ld % 4 != 0 || (reinterpret_cast<uintptr_t>(out) & 15) != 0) return cudaErrorInvalidValue;
    BatchTables bt{};
    bt.g_rowscale = rowscale;
    bt.g_bias = bias;
    bt.g_out = out;
    bt.g_ld = out_ld;
    bt.g_act = act;
    return launch_one<2, MODE_GEMM>(tmA, tmB, kp, nA, nB, 0.f, nullptr, nullptr, nullptr, 0, nullptr, status, timeout,
                                    0, grid, default_group_m(kp), bt, st);
}

cudaError_t launch_sim_tc_list(int kind, const CUtensorMap *tmA, const CUtensorMap *tmB, int kp, const long long *nA,
                               const long long *nB, float thr, const uint2 *tile_list,
                               const unsigned long long *tile_count, unsigned long long tile_cap, uint2 *cand,
                               uint64_t cap, unsigned long long *cand_count, unsigned *status, uint64_t timeout,
                               int grid, cudaStream_t st, int sym)
{
    BatchTables bt{};
    bt.tile_list = tile_list;
    bt.tile_count = tile_count;
    bt.tile_cap = tile_cap;
    bt.sym = sym;
    switch (kind) {
    case 0:
        return launch_one<0, MODE_LIST>(tmA, tmB, kp, nA, nB, thr, nullptr, nullptr, cand, cap, cand_count, status,
                                        timeout, 0, grid, 1, bt, st);
    case 1:
        return launch_one<1, MODE_LIST>(tmA, tmB, kp, nA, nB, thr, nullptr, nullptr, cand, cap, cand_count, status,
                                        timeout, 0, grid, 1, bt, st);
    case 2:
        return launch_one<2, MODE_LIST>(tmA, tmB, kp, nA, nB, thr, nullptr, nullptr, cand, cap, cand_count, status,
                                        timeout, 0, grid, 1, bt, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ej
