// Device sort of result records by (i, j): EJOIN_FLAG_SORT.
//
// The operator's result is a set of tuples (Sec. III-C); the paper fixes no
// order (Sec. IV-C keeps the pairs as a sparse matrix of offsets).  With the
// flag, the records {i, j, sim} are returned in ascending lexicographic order
// of (i, j), the order of a plain nested loop over R then S.  The sort is a
// least-significant-digit radix sort with 8-bit digits: first over the
// significant bits of j, then over those of i.  Every pass is stable, so
// after the last one the order is lexicographic.  A pass is a per-block
// digit histogram (digit-major table), a scan of that table, and a stable
// scatter: inside a block the items are ranked in order with warp matching
// and a per-round table of warp counts.
#include <algorithm>

#include "ejoin_internal.cuh"

namespace ej {

namespace {
constexpr int ST_THREADS = 256;
constexpr int ST_WARPS = ST_THREADS / 32;
constexpr int ST_ROUNDS = 16;
constexpr int ST_TILE = ST_THREADS * ST_ROUNDS;  // records per block
constexpr int SCAN_T = 1024;
constexpr int SCAN_ITEMS_T = SCAN_T * 8;

__device__ __forceinline__ unsigned digit_of(const ejoin_pair &p, int part, int shift)
{
    return ((part ? p.i : p.j) >> shift) & 0xffu;
}

// counts[d * nblocks + b] = records of block b with digit d
__global__ void __launch_bounds__(ST_THREADS) sort_hist_kernel(const ejoin_pair *__restrict__ in, uint32_t n,
                                                               int part, int shift, uint32_t *counts)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t b0 = (uint64_t)blockIdx.x * ST_TILE;
    for (int r = 0; r < ST_ROUNDS; ++r) {
        const uint64_t k = b0 + (uint64_t)r * ST_THREADS + threadIdx.x;
        if (k < n) atomicAdd(&h[digit_of(in[k], part, shift)], 1u);
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Block-wide inclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_scan1(uint32_t &x)
{
    __shared__ uint32_t w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t a = lane < (int)(blockDim.x >> 5) ? w[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, a, o);
            if (lane >= o) a += y;
        }
        w[lane] = a;
    }
    __syncthreads();
    if (warp) x += w[warp - 1];
    const uint32_t tot = w[(blockDim.x >> 5) - 1];
    __syncthreads();
    return tot;
}

// Exclusive scan of m values in place, three phases (SCAN_ITEMS_T values per block).
__global__ void __launch_bounds__(SCAN_T) sort_scan_reduce_kernel(const uint32_t *__restrict__ v, uint64_t m,
                                                                  uint32_t *tot)
{
    const uint64_t b0 = (uint64_t)blockIdx.x * SCAN_ITEMS_T;
    uint32_t a = 0;
    for (int k = threadIdx.x; k < SCAN_ITEMS_T; k += SCAN_T)
        if (b0 + k < m) a += v[b0 + k];
    const uint32_t t = block_scan1(a);
    if (threadIdx.x == 0) tot[blockIdx.x] = t;
}

__global__ void __launch_bounds__(SCAN_T) sort_scan_top_kernel(uint32_t *tot, int blocks)
{
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < blocks; base += SCAN_T) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < blocks ? tot[i] : 0u;
        uint32_t x = v;
        const uint32_t t = block_scan1(x);
        if (i < blocks) tot[i] = carry + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += t;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SCAN_T) sort_scan_down_kernel(uint32_t *v, uint64_t m, const uint32_t *tot)
{
    constexpr int PER = SCAN_ITEMS_T / SCAN_T;
    const uint64_t i0 = (uint64_t)blockIdx.x * SCAN_ITEMS_T + (uint64_t)threadIdx.x * PER;
    uint32_t x[PER], s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        x[k] = i0 + k < m ? v[i0 + k] : 0u;
        s += x[k];
    }
    uint32_t incl = s;
    block_scan1(incl);
    uint32_t run = tot[blockIdx.x] + incl - s;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (i0 + k < m) v[i0 + k] = run;
        run += x[k];
    }
}

// Stable scatter: the records of block b with digit d go to out[offs[d * nblocks + b] + their rank among
// the block's records with digit d, in input order].
__global__ void __launch_bounds__(ST_THREADS) sort_scatter_kernel(const ejoin_pair *__restrict__ in, uint32_t n,
                                                                  int part, int shift,
                                                                  const uint32_t *__restrict__ offs,
                                                                  ejoin_pair *__restrict__ out)
{
    __shared__ uint32_t base[256];             // this block's next position per digit
    __shared__ uint32_t wc[ST_WARPS][256];     // this round: records per (warp, digit)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offs[(uint64_t)threadIdx.x * gridDim.x + blockIdx.x];
    const uint64_t b0 = (uint64_t)blockIdx.x * ST_TILE;
    for (int r = 0; r < ST_ROUNDS; ++r) {
        // items of a round are in order (warp, lane): rank = (earlier warps, same digit) + (earlier lanes)
        for (int w = 0; w < ST_WARPS; ++w) wc[w][threadIdx.x] = 0u;
        __syncthreads();
        const uint64_t k = b0 + (uint64_t)r * ST_THREADS + threadIdx.x;
        const bool ok = k < n;
        ejoin_pair p{};
        unsigned dg = 256u + (unsigned)lane;  // distinct dummy keys for lanes without a record
        if (ok) {
            p = in[k];
            dg = digit_of(p, part, shift);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const unsigned before = __popc(peers & ((1u << lane) - 1u));
        if (ok && before == 0) wc[warp][dg] = (uint32_t)__popc(peers);
        __syncthreads();
        // per digit (thread = digit): exclusive prefix over the warps, then advance the block's base
        {
            uint32_t run = 0;
            for (int w = 0; w < ST_WARPS; ++w) {
                const uint32_t c = wc[w][threadIdx.x];
                wc[w][threadIdx.x] = run;
                run += c;
            }
            // base[] is read below for this round's writes, so the advance is applied after them
            __syncthreads();
            if (ok) out[base[dg] + wc[warp][dg] + before] = p;
            __syncthreads();
            base[threadIdx.x] += run;
        }
        __syncthreads();
    }
}

}  // namespace

size_t sort_pairs_scratch_bytes(uint64_t n)
{
    const uint64_t nb = std::max<uint64_t>(1, (n + ST_TILE - 1) / ST_TILE);
    const uint64_t m = 256 * nb;
    const uint64_t sb = (m + SCAN_ITEMS_T - 1) / SCAN_ITEMS_T;
    return (size_t)(m + sb + 1) * sizeof(uint32_t);
}

cudaError_t launch_sort_pairs(ejoin_pair *data, ejoin_pair *tmp, uint64_t n, uint64_t n_i, uint64_t n_j,
                              void *scratch, cudaStream_t st)
{
    if (n <= 1) return cudaSuccess;
    if (n > 0xffffffffull || !data || !tmp || !scratch) return cudaErrorInvalidValue;
    auto bits = [](uint64_t range) {
        int b = 0;
        while (b < 32 && (range - 1) >> b) ++b;
        return b;
    };
    const int bj = bits(std::max<uint64_t>(n_j, 1)), bi = bits(std::max<uint64_t>(n_i, 1));
    const uint32_t nb = (uint32_t)((n + ST_TILE - 1) / ST_TILE);
    const uint64_t m = 256ull * nb;
    const uint32_t sb = (uint32_t)((m + SCAN_ITEMS_T - 1) / SCAN_ITEMS_T);
    uint32_t *counts = static_cast<uint32_t *>(scratch);
    uint32_t *tot = counts + m;
    ejoin_pair *src = data, *dst = tmp;
    int passes = 0;
    for (int part = 0; part < 2; ++part) {
        const int b = part ? bi : bj;
        for (int shift = 0; shift < b; shift += 8) {
            sort_hist_kernel<<<nb, ST_THREADS, 0, st>>>(src, (uint32_t)n, part, shift, counts);
            sort_scan_reduce_kernel<<<sb, SCAN_T, 0, st>>>(counts, m, tot);
            sort_scan_top_kernel<<<1, SCAN_T, 0, st>>>(tot, (int)sb);
            sort_scan_down_kernel<<<sb, SCAN_T, 0, st>>>(counts, m, tot);
            sort_scatter_kernel<<<nb, ST_THREADS, 0, st>>>(src, (uint32_t)n, part, shift, counts, dst);
            std::swap(src, dst);
            ++passes;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (passes & 1) e = cudaMemcpyAsync(data, src, n * sizeof(ejoin_pair), cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace ej
