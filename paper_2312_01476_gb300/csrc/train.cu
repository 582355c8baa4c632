// Device steps of the sketch network's training set-up (ejoin_sketch_train):
// seeded parameter initialisation, the labelled pair set drawn from the exact
// join of a held-out sample plus random pairs, the shuffled order of every
// epoch, and the records whose sort gives the calibration quantile.  The paper
// has no learned component; these kernels only prepare data for the training
// kernels of mlp.cu.
//
// Randomness is counter-based: every draw is a function of (seed, stream tag,
// index) through the SplitMix64 finaliser, so a result depends on the seed
// only, not on the launch configuration.
#include <algorithm>

#include "mlp_internal.cuh"

namespace ej {

namespace {

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    // SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", 2014)
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t seed, uint64_t tag, uint64_t k)
{
    return mix64(seed ^ mix64(tag ^ mix64(k)));
}

// Standard normal from two uniform draws (Box-Muller).
__device__ __forceinline__ float normal(uint64_t seed, uint64_t tag, uint64_t k)
{
    const uint64_t r = draw(seed, tag, k);
    const float u1 = ((float)(uint32_t)(r >> 40) + 0.5f) * (1.0f / 16777216.0f);  // (0, 1)
    const float u2 = (float)(uint32_t)(r & 0xffffffu) * (1.0f / 16777216.0f);     // [0, 1)
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

__global__ void init_params_kernel(float *params, int64_t n_w1, int64_t n_b1, int64_t n_w2, int64_t n_b2,
                                   float s1, float s2, uint64_t seed)
{
    const int64_t n = n_w1 + n_b1 + n_w2 + n_b2;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (k < n_w1) v = s1 * normal(seed, 1, (uint64_t)k);
        else if (k >= n_w1 + n_b1 && k < n_w1 + n_b1 + n_w2) v = s2 * normal(seed, 2, (uint64_t)k);
        params[k] = v;
    }
}

constexpr int LB_THREADS = 256;
constexpr int LB_ITEMS = 16;
constexpr int LB_TILE = LB_THREADS * LB_ITEMS;

// A join pair (i, j), i != j, is kept iff its draw falls below keep (a fraction of 2^32).
__device__ __forceinline__ bool keep_pair(const ejoin_pair &p, uint64_t seed, uint32_t keep)
{
    return p.i != p.j && (uint32_t)(draw(seed, 3, ((uint64_t)p.i << 32) | p.j) >> 32) < keep;
}

__global__ void __launch_bounds__(LB_THREADS) label_count_kernel(const ejoin_pair *__restrict__ pairs, uint64_t n,
                                                                 uint64_t seed, uint32_t keep, uint32_t *counts)
{
    __shared__ uint32_t s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * LB_TILE + (uint64_t)threadIdx.x * LB_ITEMS;
    uint32_t c = 0;
    for (int k = 0; k < LB_ITEMS; ++k)
        if (base + k < n && keep_pair(pairs[base + k], seed, keep)) ++c;
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

// one block: exclusive scan of nb counts in place; total into *total
__global__ void __launch_bounds__(1024) label_scan_kernel(uint32_t *counts, int64_t nb, unsigned long long *total)
{
    __shared__ uint32_t w[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        const uint32_t v = i < nb ? counts[i] : 0u;
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
        const uint32_t excl = (warp ? w[warp - 1] : 0u) + x - v;
        if (i < nb) counts[i] = (uint32_t)carry + excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += w[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Kept pairs in input order: p, q, their exact similarity as target, weight w_join.
__global__ void __launch_bounds__(LB_THREADS) label_scatter_kernel(const ejoin_pair *__restrict__ pairs, uint64_t n,
                                                                   uint64_t seed, uint32_t keep,
                                                                   const uint32_t *__restrict__ offs, float w_join,
                                                                   uint64_t cap, uint32_t *p, uint32_t *q, float *t,
                                                                   float *w)
{
    __shared__ uint32_t wsum[LB_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * LB_TILE + (uint64_t)threadIdx.x * LB_ITEMS;
    uint32_t c = 0;
    for (int k = 0; k < LB_ITEMS; ++k)
        if (base + k < n && keep_pair(pairs[base + k], seed, keep)) ++c;
    // exclusive rank of this thread's first kept pair inside the block (threads in order)
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int v = 0; v < warp; ++v) before += wsum[v];
    uint32_t pos = offs[blockIdx.x] + before + x - c;
    for (int k = 0; k < LB_ITEMS; ++k) {
        if (base + k < n) {
            const ejoin_pair pr = pairs[base + k];
            if (keep_pair(pr, seed, keep) && pos < cap) {
                p[pos] = pr.i;
                q[pos] = pr.j;
                t[pos] = pr.sim;
                w[pos] = w_join;
                ++pos;
            }
        }
    }
}

__global__ void random_pairs_kernel(uint32_t *p, uint32_t *q, float *w, int64_t n_pairs, uint32_t n_rows,
                                    uint64_t seed)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pairs;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r = draw(seed, 4, (uint64_t)k);
        p[k] = (uint32_t)(((r >> 32) * (uint64_t)n_rows) >> 32);
        q[k] = (uint32_t)(((r & 0xffffffffull) * (uint64_t)n_rows) >> 32);
        w[k] = 1.f;
    }
}

// A bijection of [0, n) (balanced Feistel network over 2 h bits, 4 rounds, with cycle walking), keyed
// by (seed, epoch): the order in which an epoch visits the labelled pairs.
struct Perm {
    uint64_t n;
    int h;          // half width in bits
    uint64_t key;
};

__device__ __forceinline__ uint64_t perm_at(const Perm &pm, uint64_t x)
{
    const uint64_t mask = (1ull << pm.h) - 1ull;
    do {
        uint64_t l = x >> pm.h, r = x & mask;
#pragma unroll
        for (int round = 0; round < 4; ++round) {
            const uint64_t f = mix64(pm.key ^ ((uint64_t)round << 56) ^ r) & mask;
            const uint64_t nl = r;
            r = l ^ f;
            l = nl;
        }
        x = (l << pm.h) | r;
    } while (x >= pm.n);
    return x;
}

__global__ void gather_batch_kernel(const uint32_t *__restrict__ p, const uint32_t *__restrict__ q,
                                    const float *__restrict__ t, const float *__restrict__ w, Perm pm, uint64_t b0,
                                    int64_t m, uint32_t *bp, uint32_t *bq, float *bt, float *bw)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t s = perm_at(pm, b0 + (uint64_t)k);
        bp[k] = p[s];
        bq[k] = q[s];
        bt[k] = t[s];
        bw[k] = w[s];
    }
}

// rec[k] = {f2ord(v[k]), k, v[k]}: sorted by (i, j), the records give the values in ascending order
__global__ void value_records_kernel(const float *__restrict__ v, int64_t n, ejoin_pair *rec)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        rec[k] = ejoin_pair{f2ord(v[k]), (uint32_t)k, v[k]};
}

__global__ void inverse_perm_kernel(const uint32_t *__restrict__ perm, int64_t n, uint32_t *inv)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        inv[perm[k]] = (uint32_t)k;
}

__global__ void tile_bitmap_kernel(const uint2 *__restrict__ list, const unsigned long long *__restrict__ count,
                                   uint64_t cap, int64_t tB, uint32_t *bits)
{
    uint64_t n = *count;
    if (n > cap) n = cap;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = (uint64_t)list[k].x * (uint64_t)tB + list[k].y;
        atomicOr(bits + (b >> 5), 1u << (b & 31));
    }
}

__device__ __forceinline__ bool bit_at(const uint32_t *bits, uint64_t b) { return (bits[b >> 5] >> (b & 31)) & 1u; }

// For each exact match (i', j) of the sampled rows (R row i' * stride) with S: is its tile pair kept?
__global__ void recall_count_kernel(const ejoin_pair *__restrict__ pairs, uint64_t n, uint32_t stride,
                                    const uint32_t *__restrict__ invA, const uint32_t *__restrict__ invB,
                                    const uint32_t *__restrict__ bits, int64_t tB, int sym, unsigned long long *found)
{
    unsigned long long f = 0;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = invA[(uint64_t)pairs[k].i * stride], b = invB[pairs[k].j];
        bool kept = bit_at(bits, (a >> 7) * (uint64_t)tB + (b >> 8));
        if (sym) kept = kept || bit_at(bits, (b >> 7) * (uint64_t)tB + (a >> 8));
        f += kept ? 1ull : 0ull;
    }
    f = __reduce_add_sync(0xffffffffu, (unsigned)f);
    if ((threadIdx.x & 31) == 0 && f) atomicAdd(found, f);
}

unsigned grid_for(int64_t n, int num_sms)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8));
}

}  // namespace

cudaError_t launch_init_params(float *params, int d, int hid, int out, uint64_t seed, int num_sms, cudaStream_t st)
{
    const int64_t n1 = (int64_t)hid * d, n2 = (int64_t)out * hid;
    init_params_kernel<<<grid_for(n1 + hid + n2 + out, num_sms), 256, 0, st>>>(
        params, n1, hid, n2, out, 1.0f / sqrtf((float)d), 1.0f / sqrtf((float)hid), seed);
    return cudaGetLastError();
}

size_t label_scratch_bytes(uint64_t n_join)
{
    // a multiple of 16 bytes, so that a caller may place 8-byte counters right after it
    const uint64_t nb = std::max<uint64_t>(1, (n_join + LB_TILE - 1) / LB_TILE);
    return (size_t)((nb * 4 + 15) / 16 * 16);
}

cudaError_t launch_label_join_pairs(const ejoin_pair *pairs, uint64_t n, uint64_t seed, uint32_t keep, float w_join,
                                    void *scratch, unsigned long long *d_total, uint64_t cap, uint32_t *p, uint32_t *q,
                                    float *t, float *w, cudaStream_t st)
{
    if (n == 0) return cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), st);
    const int64_t nb = (int64_t)((n + LB_TILE - 1) / LB_TILE);
    uint32_t *counts = static_cast<uint32_t *>(scratch);
    label_count_kernel<<<(unsigned)nb, LB_THREADS, 0, st>>>(pairs, n, seed, keep, counts);
    label_scan_kernel<<<1, 1024, 0, st>>>(counts, nb, d_total);
    label_scatter_kernel<<<(unsigned)nb, LB_THREADS, 0, st>>>(pairs, n, seed, keep, counts, w_join, cap, p, q, t,
                                                              w);
    return cudaGetLastError();
}

cudaError_t launch_random_pairs(uint32_t *p, uint32_t *q, float *w, int64_t n_pairs, uint32_t n_rows, uint64_t seed,
                                int num_sms, cudaStream_t st)
{
    if (n_pairs <= 0) return cudaSuccess;
    random_pairs_kernel<<<grid_for(n_pairs, num_sms), 256, 0, st>>>(p, q, w, n_pairs, n_rows, seed);
    return cudaGetLastError();
}

cudaError_t launch_gather_batch(const uint32_t *p, const uint32_t *q, const float *t, const float *w, uint64_t n,
                                uint64_t seed, int epoch, uint64_t b0, int64_t m, uint32_t *bp, uint32_t *bq,
                                float *bt, float *bw, int num_sms, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    Perm pm;
    pm.n = n;
    int bits = 2;
    while (bits < 62 && (1ull << bits) < n) bits += 2;  // 2 h bits cover [0, n); walks stay short (< 4 n)
    pm.h = bits / 2;
    pm.key = mix64(seed ^ 0x5eedull) ^ mix64((uint64_t)epoch + 17);
    gather_batch_kernel<<<grid_for(m, num_sms), 256, 0, st>>>(p, q, t, w, pm, b0, m, bp, bq, bt, bw);
    return cudaGetLastError();
}

cudaError_t launch_value_records(const float *v, int64_t n, ejoin_pair *rec, int num_sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    value_records_kernel<<<grid_for(n, num_sms), 256, 0, st>>>(v, n, rec);
    return cudaGetLastError();
}

cudaError_t launch_recall_probe(const uint32_t *permA, int64_t nA, const uint32_t *permB, int64_t nB,
                                const uint2 *list, const unsigned long long *list_count, uint64_t list_cap,
                                int64_t tA, int64_t tB, const ejoin_pair *pairs, uint64_t n_pairs, uint32_t stride,
                                int sym, void *scratch, unsigned long long *found, int num_sms, cudaStream_t st)
{
    uint32_t *invA = static_cast<uint32_t *>(scratch);
    uint32_t *invB = invA + nA;
    uint32_t *bits = invB + nB;
    const uint64_t words = ((uint64_t)tA * (uint64_t)tB + 31) / 32;
    cudaError_t e = cudaMemsetAsync(bits, 0, words * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(found, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    inverse_perm_kernel<<<grid_for(nA, num_sms), 256, 0, st>>>(permA, nA, invA);
    inverse_perm_kernel<<<grid_for(nB, num_sms), 256, 0, st>>>(permB, nB, invB);
    tile_bitmap_kernel<<<grid_for((int64_t)std::max<uint64_t>(list_cap, 1), num_sms), 256, 0, st>>>(
        list, list_count, list_cap, tB, bits);
    if (n_pairs)
        recall_count_kernel<<<grid_for((int64_t)n_pairs, num_sms), 256, 0, st>>>(pairs, n_pairs, stride, invA, invB,
                                                                                  bits, tB, sym, found);
    return cudaGetLastError();
}

size_t recall_probe_scratch_bytes(int64_t nA, int64_t nB, int64_t tA, int64_t tB)
{
    // a multiple of 16 bytes, so that a caller may place 8-byte counters right after it
    const size_t b = (size_t)(nA + nB) * 4 + (((size_t)tA * (size_t)tB + 31) / 32) * 4;
    return (b + 15) / 16 * 16;
}

}  // namespace ej
