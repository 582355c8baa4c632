// Batched E-joins: many independent joins (uneven, post-selection sizes) in
// one persistent contraction launch, captured once in a CUDA graph.
//
// Every job is the operator of Sec. III-C (Eq. (E-theta-Join)) with its own
// threshold.  The rows of all jobs' R (and S) are normalised into one
// concatenated operand each, so one pair of TMA tensor maps covers the whole
// batch; a device job table maps the global tile space onto (job, row tile,
// column tile) (tiles of different jobs are independent blocks of the
// decomposition of Eq. (Block Matrix Dot Product Decomposition)).  A sizing
// run fixes the candidate and pair buffers, an optional autotuner picks the
// raster width of the contraction, and the whole sequence (counter reset,
// two normalisations, contraction, re-score) is captured into a CUDA graph
// that later runs replay without any host synchronisation.
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "host_internal.h"

using namespace ej;
using namespace ej::host;

struct ejoin_batch {
    ejoin_ctx *ctx = nullptr;
    int device = 0;  // the context's device, kept for teardown
    int n_jobs = 0;
    int d = 0;
    int64_t kp = 0;
    int fmt = FMT_BF16;
    int kind = 0;
    float band = 0.f;
    int group_m = 16;
    float ms_normalize = 0.f, ms_contract = 0.f, ms_rescore = 0.f;  // stage split of one eager run at plan time
    uint32_t flags = 0;
    // device tables
    Buf tile_off, a_off, b_off, nA, nB, thr, eps, xR, ldR, xS, ldS, rowoffA, rowoffB;
    // operands and results
    Buf A, B, invA, invB, scaleA, scaleB, misc, cand, pairs;
    // per-job selections: predicate tables of each side, the kept rows' indices among all rows, the jobs'
    // offsets among all rows, per-block counts and offsets of the compaction
    bool has_sel = false;
    Buf selA_attr, selA_op, selA_c, selA_bits, selB_attr, selB_op, selB_c, selB_bits;
    Buf allA_off, allB_off, idsA, idsB, sel_cnt, sel_off;
    // streaming re-score: the candidates sorted by (job, S block, A row), its bucket tables, the first bucket
    // of every job and the S block height
    Buf sorted, sbuf, bbase;
    bool stream = false;
    int64_t n_buckets = 0, sblock_rows = 0;
    uint64_t cand_cap = 0, pair_cap = 0;
    int64_t rowsA = 0, rowsB = 0, total_tiles = 0;
    bool aligned = false;
    CUtensorMap tmA{}, tmB{};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches_per_run = 0;
};

namespace {

constexpr int64_t STREAM_SBLOCK_BYTES = 32ll << 20;

// ------------------------------------------------------------ per-job selections
// Predicates of one side of every job (device arrays); row_off: the jobs' offsets among all of the side's
// concatenated rows (n_jobs + 1 entries).
struct JobSel {
    const int32_t *const *attr;
    const int *op;
    const int *c;
    const uint32_t *const *bits;
    const long long *row_off;
    int n_jobs;
};

// Keep flag of concatenated row g; job: a cursor that only moves forward (each thread's rows increase).
__device__ __forceinline__ bool job_keep(const JobSel &t, int64_t g, int &job)
{
    if (job < 0) {
        int lo = 0, hi = t.n_jobs;  // row_off[lo] <= g < row_off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(t.row_off + mid) <= g) lo = mid;
            else hi = mid;
        }
        job = lo;
    }
    while (__ldg(t.row_off + job + 1) <= g) ++job;
    const SelArgs s{t.attr[job], t.op[job], t.c[job], t.bits[job]};
    return sel_keep(s, g - __ldg(t.row_off + job));
}

// Rows kept per block of SEL_ROWS_PER_BLOCK concatenated rows
__global__ void __launch_bounds__(SEL_THREADS) job_sel_count_kernel(JobSel t, int64_t n, uint32_t *block_counts)
{
    __shared__ int red[SEL_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SEL_ROWS_PER_BLOCK;
    int cnt = 0, job = -1;
    for (int it = 0; it < SEL_ITEMS; ++it) {
        const int64_t g = base + (int64_t)it * SEL_THREADS + threadIdx.x;
        if (g < n && job_keep(t, g, job)) ++cnt;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) red[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < SEL_THREADS / 32; ++w) tot += red[w];
        block_counts[blockIdx.x] = (uint32_t)tot;
    }
}

// ids[k] = the k-th kept concatenated row (order-preserving)
__global__ void __launch_bounds__(SEL_THREADS) job_sel_scatter_kernel(JobSel t, int64_t n,
                                                                      const uint32_t *block_offsets, uint32_t *ids)
{
    __shared__ int wcount[SEL_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SEL_ROWS_PER_BLOCK;
    uint32_t running = block_offsets[blockIdx.x];
    int job = -1;
    for (int it = 0; it < SEL_ITEMS; ++it) {
        const int64_t g = base + (int64_t)it * SEL_THREADS + threadIdx.x;
        const bool k = g < n && job_keep(t, g, job);
        const unsigned m = __ballot_sync(0xffffffffu, k);
        if (lane == 0) wcount[warp] = __popc(m);
        __syncthreads();
        uint32_t before = 0, strip = 0;
        for (int w = 0; w < SEL_THREADS / 32; ++w) {
            const int cw = wcount[w];
            before += (w < warp) ? cw : 0;
            strip += cw;
        }
        if (k) ids[running + before + __popc(m & ((1u << lane) - 1u))] = (uint32_t)g;
        running += strip;
        __syncthreads();
    }
}

// First k with ids[k] >= g among the n kept rows (ids ascending)
__device__ __forceinline__ long long kept_before(const uint32_t *ids, long long n, long long g)
{
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((long long)__ldg(ids + mid) < g) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// The job table from the kept rows (one block): a_off / b_off (also the normalisations' row offsets), nA / nB,
// tile_off (tiles of 128 x 256) and bbase (first sort bucket: nA x max(1, ceil(nB / sblock_rows)) per job).
__global__ void __launch_bounds__(1024) job_sel_tables_kernel(const uint32_t *idsA, const uint32_t *idsB,
                                                              const long long *n_kept, const long long *allA_off,
                                                              const long long *allB_off, int n_jobs,
                                                              long long sblock_rows, long long *a_off,
                                                              long long *b_off, long long *rowoffA,
                                                              long long *rowoffB, int *nA, int *nB,
                                                              long long *tile_off, long long *bbase)
{
    __shared__ unsigned long long wt[32], wb[32];
    __shared__ unsigned long long carry_t, carry_b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long ka = n_kept[0], kb = n_kept[1];
    if (threadIdx.x == 0) carry_t = carry_b = 0ull;
    __syncthreads();
    for (int base = 0; base < n_jobs; base += 1024) {
        const int j = base + threadIdx.x;
        unsigned long long tiles = 0, bk = 0;
        if (j < n_jobs) {
            const long long a0 = kept_before(idsA, ka, allA_off[j]), a1 = kept_before(idsA, ka, allA_off[j + 1]);
            const long long b0 = kept_before(idsB, kb, allB_off[j]), b1 = kept_before(idsB, kb, allB_off[j + 1]);
            const long long na = a1 - a0, nb = b1 - b0;
            a_off[j] = rowoffA[j] = a0;
            b_off[j] = rowoffB[j] = b0;
            nA[j] = (int)na;
            nB[j] = (int)nb;
            tiles = (unsigned long long)(((na + 127) / 128) * ((nb + 255) / 256));
            const long long nsb = (nb + sblock_rows - 1) / sblock_rows;
            bk = (unsigned long long)(na * (nsb > 0 ? nsb : 1ll));
        }
        unsigned long long xt = tiles, xb = bk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long yt = __shfl_up_sync(0xffffffffu, xt, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
            if (lane >= o) {
                xt += yt;
                xb += yb;
            }
        }
        if (lane == 31) {
            wt[warp] = xt;
            wb[warp] = xb;
        }
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = wt[lane], u = wb[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long yt = __shfl_up_sync(0xffffffffu, t, o), yb = __shfl_up_sync(0xffffffffu, u, o);
                if (lane >= o) {
                    t += yt;
                    u += yb;
                }
            }
            wt[lane] = t;
            wb[lane] = u;
        }
        __syncthreads();
        if (j < n_jobs) {
            tile_off[j] = (long long)(carry_t + (warp ? wt[warp - 1] : 0ull) + xt - tiles);
            bbase[j] = (long long)(carry_b + (warp ? wb[warp - 1] : 0ull) + xb - bk);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_t += wt[31];
            carry_b += wb[31];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tile_off[n_jobs] = (long long)carry_t;
        bbase[n_jobs] = (long long)carry_b;
        a_off[n_jobs] = rowoffA[n_jobs] = ka;
        b_off[n_jobs] = rowoffB[n_jobs] = kb;
    }
}

template <typename T>
cudaError_t upload(Buf &b, const std::vector<T> &v)
{
    cudaError_t e = ensure(b, std::max<size_t>(v.size() * sizeof(T), 16));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Enqueue one run of the batch pipeline on stream st (eager or under capture).
// evs (optional, eager runs only): four events recorded before the normalisations, before the
// contraction, before the re-score and after it.
cudaError_t enqueue(ejoin_batch *b, cudaStream_t st, int group_m, bool contract_only = false,
                    cudaEvent_t *evs = nullptr)
{
    ejoin_ctx *c = b->ctx;
    DevMisc *dm = (DevMisc *)b->misc.p;
    cudaError_t e;
    if (evs) cudaEventRecord(evs[0], st);
    const uint32_t *idsA = b->has_sel ? (const uint32_t *)b->idsA.p : nullptr;
    const uint32_t *idsB = b->has_sel ? (const uint32_t *)b->idsB.p : nullptr;
    if (!contract_only) {
        if ((e = cudaMemsetAsync(dm, 0, sizeof(DevMisc), st)) != cudaSuccess) return e;
        if (b->has_sel) {
            // the kept rows of every job (order-preserving), then the job table from their counts
            const int64_t nbA = (b->rowsA + SEL_ROWS_PER_BLOCK - 1) / SEL_ROWS_PER_BLOCK;
            const int64_t nbB = (b->rowsB + SEL_ROWS_PER_BLOCK - 1) / SEL_ROWS_PER_BLOCK;
            uint32_t *cnt = (uint32_t *)b->sel_cnt.p, *offs = (uint32_t *)b->sel_off.p;
            const JobSel ta{(const int32_t *const *)b->selA_attr.p, (const int *)b->selA_op.p,
                            (const int *)b->selA_c.p, (const uint32_t *const *)b->selA_bits.p,
                            (const long long *)b->allA_off.p, b->n_jobs};
            const JobSel tb{(const int32_t *const *)b->selB_attr.p, (const int *)b->selB_op.p,
                            (const int *)b->selB_c.p, (const uint32_t *const *)b->selB_bits.p,
                            (const long long *)b->allB_off.p, b->n_jobs};
            if (nbA > 0) {
                job_sel_count_kernel<<<(unsigned)nbA, SEL_THREADS, 0, st>>>(ta, b->rowsA, cnt);
                if ((e = launch_sel_scan(cnt, nbA, offs, &dm->n_sel[0], st)) != cudaSuccess) return e;
                job_sel_scatter_kernel<<<(unsigned)nbA, SEL_THREADS, 0, st>>>(ta, b->rowsA, offs, (uint32_t *)b->idsA.p);
            }
            if (nbB > 0) {
                job_sel_count_kernel<<<(unsigned)nbB, SEL_THREADS, 0, st>>>(tb, b->rowsB, cnt + nbA);
                if ((e = launch_sel_scan(cnt + nbA, nbB, offs + nbA, &dm->n_sel[1], st)) != cudaSuccess) return e;
                job_sel_scatter_kernel<<<(unsigned)nbB, SEL_THREADS, 0, st>>>(tb, b->rowsB, offs + nbA,
                                                                              (uint32_t *)b->idsB.p);
            }
            job_sel_tables_kernel<<<1, 1024, 0, st>>>(
                idsA, idsB, dm->n_sel, (const long long *)b->allA_off.p, (const long long *)b->allB_off.p, b->n_jobs,
                b->sblock_rows, (long long *)b->a_off.p, (long long *)b->b_off.p, (long long *)b->rowoffA.p,
                (long long *)b->rowoffB.p, (int *)b->nA.p, (int *)b->nB.p, (long long *)b->tile_off.p,
                (long long *)b->bbase.p);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if ((e = launch_normalize_batch(b->fmt, (const float *const *)b->xR.p, (const long long *)b->ldR.p,
                                        (const long long *)b->rowoffA.p, b->n_jobs, b->rowsA, b->d, b->A.p,
                                        (int)b->kp, (float *)b->invA.p, (float *)b->scaleA.p, &dm->status,
                                        c->num_sms, st, b->aligned, idsA, (const long long *)b->allA_off.p)) !=
            cudaSuccess)
            return e;
        if ((e = launch_normalize_batch(b->fmt, (const float *const *)b->xS.p, (const long long *)b->ldS.p,
                                        (const long long *)b->rowoffB.p, b->n_jobs, b->rowsB, b->d, b->B.p,
                                        (int)b->kp, (float *)b->invB.p, (float *)b->scaleB.p, &dm->status,
                                        c->num_sms, st, b->aligned, idsB, (const long long *)b->allB_off.p)) !=
            cudaSuccess)
            return e;
    } else {
        if ((e = cudaMemsetAsync(&dm->cand_count, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    }
    if (evs) cudaEventRecord(evs[1], st);
    BatchTables bt{(const long long *)b->tile_off.p, (const long long *)b->a_off.p, (const long long *)b->b_off.p,
                   (const int *)b->nA.p, (const int *)b->nB.p, (const float *)b->thr.p, b->n_jobs};
    if ((e = launch_sim_tc_batch(b->kind, &b->tmA, &b->tmB, (int)b->kp, bt, (const float *)b->scaleA.p,
                                 (const float *)b->scaleB.p, (uint2 *)b->cand.p, b->cand_cap, &dm->cand_count,
                                 &dm->status, c->timeout, c->num_sms, group_m, st)) != cudaSuccess)
        return e;
    if (contract_only) return cudaSuccess;
    if (evs) cudaEventRecord(evs[2], st);
    BatchRows br{(const float *const *)b->xR.p, (const long long *)b->ldR.p, (const float *const *)b->xS.p,
                 (const long long *)b->ldS.p, (const long long *)b->a_off.p, (const long long *)b->b_off.p,
                 (const float *)b->eps.p, b->n_jobs, idsA, idsB, (const long long *)b->allA_off.p,
                 (const long long *)b->allB_off.p};
    if (b->stream)
        e = launch_rescore_stream_batch((const uint2 *)b->cand.p, &dm->cand_count, b->cand_cap, (uint2 *)b->sorted.p,
                                        b->sbuf.p, b->rowsA, br, (const long long *)b->bbase.p, (const int *)b->nA.p,
                                        b->n_buckets, b->sblock_rows, b->d, (const float *)b->invA.p,
                                        (const float *)b->invB.p, c->fp64_band, (BatchPair *)b->pairs.p, b->pair_cap,
                                        &dm->pair_count, &dm->band_count, c->num_sms, st);
    else
        e = launch_rescore_batch((const uint2 *)b->cand.p, &dm->cand_count, b->cand_cap, br, b->d,
                                 (const float *)b->invA.p, (const float *)b->invB.p, c->fp64_band,
                                 (BatchPair *)b->pairs.p, b->pair_cap, &dm->pair_count, &dm->band_count, b->aligned,
                                 c->num_sms, st);
    if (evs) cudaEventRecord(evs[3], st);
    return e;
}

ejoin_status read_misc(ejoin_batch *b, DevMisc &hm, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(&hm, b->misc.p, sizeof(DevMisc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    if (hm.status & ERR_NONFINITE) return EJOIN_ENONFINITE;
    if (hm.status & ERR_TIMEOUT) return EJOIN_ETIMEOUT;
    if (hm.status) return EJOIN_ECUDA;
    return EJOIN_OK;
}

// ---------------------------------------------------------------- autotuner
// Cache of the fastest raster width per size class, in memory and (when the
// environment variable EJOIN_TUNE_FILE names a file) on disk, one
// "key value" line per entry.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("EJOIN_TUNE_FILE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[256];
    int v;
    while (std::fscanf(f, "%255s %d", key, &v) == 2) g_tune[key] = v;
    std::fclose(f);
}

void tune_store()
{
    const char *path = std::getenv("EJOIN_TUNE_FILE");
    if (!path) return;
    FILE *f = std::fopen(path, "w");
    if (!f) return;
    for (auto &kv : g_tune) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    std::fclose(f);
}

std::string size_class(const ejoin_batch *b)
{
    // kind, padded dim, log2 of jobs and of mean tiles per job
    auto lg = [](double x) { return x < 1 ? 0 : (int)std::floor(std::log2(x)); };
    char k[128];
    std::snprintf(k, sizeof k, "batch:k%d:d%lld:j%d:t%d", b->kind, (long long)b->kp, lg(b->n_jobs),
                  lg((double)b->total_tiles / std::max(1, b->n_jobs)));
    return k;
}

ejoin_status autotune(ejoin_batch *b)
{
    const std::string key = size_class(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            b->group_m = it->second;
            return EJOIN_OK;
        }
    }
    ejoin_ctx *c = b->ctx;
    const int cands[] = {4, 8, 16, 32, 64, 128};
    float best = 1e30f;
    int best_g = b->group_m;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return EJOIN_ECUDA;
    for (int g : cands) {
        float ms_sum = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, c->stream);
            if (enqueue(b, c->stream, g, true) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return EJOIN_ECUDA;
            }
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep) ms_sum += ms;  // first repetition warms caches
        }
        if (ms_sum < best) {
            best = ms_sum;
            best_g = g;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->group_m = best_g;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best_g;
    tune_store();
    return EJOIN_OK;
}

void destroy_batch(ejoin_batch *b)
{
    if (!b) return;
    // the context may already be gone: wait for the device, not for its stream
    DeviceGuard g(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (Buf *x : {&b->tile_off, &b->a_off, &b->b_off, &b->nA, &b->nB, &b->thr, &b->eps, &b->xR, &b->ldR, &b->xS,
                   &b->ldS, &b->rowoffA, &b->rowoffB, &b->A, &b->B, &b->invA, &b->invB, &b->scaleA, &b->scaleB,
                   &b->misc, &b->cand, &b->pairs, &b->sorted, &b->sbuf, &b->bbase, &b->selA_attr,
                   &b->selA_op, &b->selA_c, &b->selA_bits, &b->selB_attr, &b->selB_op, &b->selB_c, &b->selB_bits,
                   &b->allA_off, &b->allB_off, &b->idsA, &b->idsB, &b->sel_cnt, &b->sel_off})
        release(*x);
    delete b;
}

}  // namespace

extern "C" {

ejoin_status ejoin_batch_create(ejoin_ctx *c, const ejoin_job *jobs, int32_t n_jobs, uint32_t flags,
                                ejoin_batch **out)
{
    return ejoin_batch_create_sel(c, jobs, nullptr, n_jobs, flags, out);
}

ejoin_status ejoin_batch_create_sel(ejoin_ctx *c, const ejoin_job *jobs, const ejoin_job_sel *sels, int32_t n_jobs,
                                    uint32_t flags, ejoin_batch **out)
{
    if (!c || !out || n_jobs < 1 || !jobs) return EJOIN_EINVAL;
    bool has_sel = false;
    if (sels) {
        for (int j = 0; j < n_jobs; ++j) {
            for (const ejoin_sel *q : {&sels[j].R, &sels[j].S}) {
                if (q->attr && (q->op < EJOIN_LT || q->op > EJOIN_NE)) return EJOIN_EINVAL;
                if (q->attr || q->bits) has_sel = true;
            }
        }
    }
    *out = nullptr;
    if (c->prec == EJOIN_F32) return EJOIN_EUNSUPPORTED;  // the batched contraction runs on tensor cores
    const int d = jobs[0].R.d;
    int64_t sumA = 0, sumB = 0;
    bool aligned = d % 4 == 0;
    for (int j = 0; j < n_jobs; ++j) {
        const ejoin_job &jb = jobs[j];
        for (const ejoin_rel *r : {&jb.R, &jb.S}) {
            if (r->d != d || r->d < 1 || r->d > 4096 || r->n < 0 || r->n > 0x7FFFFEFF || r->ld < r->d ||
                (r->n > 0 && !r->x))
                return EJOIN_EINVAL;
            if ((reinterpret_cast<uintptr_t>(r->x) & 15) || (r->ld & 3)) aligned = false;
        }
        if (std::isnan(jb.eps)) return EJOIN_EINVAL;
        sumA += jb.R.n;
        sumB += jb.S.n;
    }
    if (sumA > 0xFFFFFEFFll || sumB > 0xFFFFFEFFll) return EJOIN_EINVAL;  // concatenated rows index with u32
    DeviceGuard g(c->device);
    ejoin_batch *b = new (std::nothrow) ejoin_batch();
    if (!b) return EJOIN_ENOMEM;
    b->ctx = c;
    b->device = c->device;
    b->n_jobs = n_jobs;
    b->d = d;
    b->flags = flags;
    b->fmt = fmt_of(c->prec);
    b->kind = c->prec == EJOIN_BF16 ? 0 : (c->prec == EJOIN_FP8_E4M3 ? 1 : 2);
    b->kp = ejoin_padded_dim(c->prec, d);
    b->band = c->band_cfg >= 0.f ? c->band_cfg : default_band(c->prec, b->kp);
    b->group_m = c->group_m > 0 ? c->group_m : 16;
    b->aligned = aligned;
    b->rowsA = sumA;
    b->rowsB = sumB;
    b->has_sel = has_sel;
    b->sblock_rows = std::max<int64_t>(1, STREAM_SBLOCK_BYTES / ((int64_t)((d + 3) / 4) * 16));

    // host tables
    std::vector<long long> tile_off(n_jobs + 1), a_off(n_jobs + 1), b_off(n_jobs + 1), ldR(n_jobs), ldS(n_jobs);
    std::vector<int> nA(n_jobs), nB(n_jobs);
    std::vector<float> thr(n_jobs), eps(n_jobs);
    std::vector<const float *> xR(n_jobs), xS(n_jobs);
    long long t = 0, ra = 0, rb = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const ejoin_job &jb = jobs[j];
        tile_off[j] = t;
        a_off[j] = ra;
        b_off[j] = rb;
        t += ((jb.R.n + 127) / 128) * ((jb.S.n + 255) / 256);
        ra += jb.R.n;
        rb += jb.S.n;
        nA[j] = (int)jb.R.n;
        nB[j] = (int)jb.S.n;
        eps[j] = jb.eps;
        thr[j] = jb.eps - b->band;
        xR[j] = jb.R.x;
        xS[j] = jb.S.x;
        ldR[j] = jb.R.ld;
        ldS[j] = jb.S.ld;
    }
    tile_off[n_jobs] = t;
    a_off[n_jobs] = ra;
    b_off[n_jobs] = rb;
    b->total_tiles = t;
    cudaError_t e = cudaSuccess;
    ejoin_status st = EJOIN_OK;
    auto fail = [&](ejoin_status s) {
        destroy_batch(b);
        return s;
    };
    if ((e = upload(b->tile_off, tile_off)) || (e = upload(b->a_off, a_off)) || (e = upload(b->b_off, b_off)) ||
        (e = upload(b->nA, nA)) || (e = upload(b->nB, nB)) || (e = upload(b->thr, thr)) ||
        (e = upload(b->eps, eps)) || (e = upload(b->xR, xR)) || (e = upload(b->xS, xS)) ||
        (e = upload(b->ldR, ldR)) || (e = upload(b->ldS, ldS)) || (e = upload(b->rowoffA, a_off)) ||
        (e = upload(b->rowoffB, b_off)))
        return fail(from_cuda(e));
    if (has_sel) {
        // predicate tables of both sides and the compaction's work arrays
        std::vector<const int32_t *> aA(n_jobs), aB(n_jobs);
        std::vector<const uint32_t *> bA(n_jobs), bB(n_jobs);
        std::vector<int> oA(n_jobs), oB(n_jobs), cA(n_jobs), cB(n_jobs);
        for (int j = 0; j < n_jobs; ++j) {
            aA[j] = sels[j].R.attr, oA[j] = sels[j].R.op, cA[j] = sels[j].R.c, bA[j] = sels[j].R.bits;
            aB[j] = sels[j].S.attr, oB[j] = sels[j].S.op, cB[j] = sels[j].S.c, bB[j] = sels[j].S.bits;
        }
        const int64_t nbA = (sumA + SEL_ROWS_PER_BLOCK - 1) / SEL_ROWS_PER_BLOCK;
        const int64_t nbB = (sumB + SEL_ROWS_PER_BLOCK - 1) / SEL_ROWS_PER_BLOCK;
        std::vector<long long> bbase0(n_jobs + 1, 0);
        if ((e = upload(b->selA_attr, aA)) || (e = upload(b->selA_op, oA)) || (e = upload(b->selA_c, cA)) ||
            (e = upload(b->selA_bits, bA)) || (e = upload(b->selB_attr, aB)) || (e = upload(b->selB_op, oB)) ||
            (e = upload(b->selB_c, cB)) || (e = upload(b->selB_bits, bB)) || (e = upload(b->allA_off, a_off)) ||
            (e = upload(b->allB_off, b_off)) || (e = upload(b->bbase, bbase0)) ||
            (e = ensure(b->idsA, (size_t)std::max<int64_t>(sumA, 4) * 4)) ||
            (e = ensure(b->idsB, (size_t)std::max<int64_t>(sumB, 4) * 4)) ||
            (e = ensure(b->sel_cnt, (size_t)std::max<int64_t>(nbA + nbB, 4) * 4)) ||
            (e = ensure(b->sel_off, (size_t)std::max<int64_t>(nbA + nbB, 4) * 4)))
            return fail(from_cuda(e));
    }
    const size_t eb = fmt_bytes(b->fmt);
    const int64_t pa = round_up(std::max<int64_t>(sumA, 1), 256), pb = round_up(std::max<int64_t>(sumB, 1), 256);
    if ((e = ensure(b->A, (size_t)pa * b->kp * eb)) || (e = ensure(b->B, (size_t)pb * b->kp * eb)) ||
        (e = ensure(b->invA, (size_t)pa * 4)) || (e = ensure(b->invB, (size_t)pb * 4)) ||
        (e = ensure(b->misc, sizeof(DevMisc))))
        return fail(from_cuda(e));
    if (b->fmt == FMT_FP8 && ((e = ensure(b->scaleA, (size_t)pa * 4)) || (e = ensure(b->scaleB, (size_t)pb * 4))))
        return fail(from_cuda(e));
    if (!make_tmap(&b->tmA, b->A.p, b->fmt, b->kp, pa, 128) || !make_tmap(&b->tmB, b->B.p, b->fmt, b->kp, pb, 256))
        return fail(EJOIN_ECUDA);

    // sizing run: candidates, then pairs
    b->cand_cap = std::max<uint64_t>(c->cap_hint, 1u << 20);
    b->pair_cap = 0;
    if ((e = ensure(b->cand, b->cand_cap * sizeof(uint2))) != cudaSuccess) return fail(from_cuda(e));
    if ((e = ensure(b->pairs, 16)) != cudaSuccess) return fail(from_cuda(e));
    DevMisc hm;
    for (int attempt = 0; attempt < 3; ++attempt) {
        if ((e = enqueue(b, c->stream, b->group_m)) != cudaSuccess) return fail(from_cuda(e));
        if ((st = read_misc(b, hm, c->stream)) != EJOIN_OK) return fail(st);
        if (hm.cand_count <= b->cand_cap) break;
        b->cand_cap = hm.cand_count + hm.cand_count / 4 + 1024;
        if ((e = ensure(b->cand, b->cand_cap * sizeof(uint2))) != cudaSuccess) return fail(from_cuda(e));
    }
    if (hm.cand_count > b->cand_cap) return fail(EJOIN_EOVERFLOW);
    if (has_sel) {
        // the tiles of the kept rows, as the last run's job table holds them
        long long tt = 0;
        if ((e = cudaMemcpy(&tt, (const long long *)b->tile_off.p + n_jobs, sizeof(tt), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
            return fail(from_cuda(e));
        b->total_tiles = tt;
    }
    b->pair_cap = std::max<uint64_t>(hm.cand_count, 1);
    if ((e = ensure(b->pairs, b->pair_cap * sizeof(BatchPair))) != cudaSuccess) return fail(from_cuda(e));
    // the re-score streams the candidates in A-row order where the rows allow it (the sizing runs above
    // gathered them in emission order)
    if (aligned && d <= 1024 && sumA > 0 && !(c->flags & EJOIN_FLAG_GATHER_RESCORE)) {
        // S blocks of about STREAM_SBLOCK_BYTES: the S rows a wave of warps reads stay in L2 while the job's
        // A rows stream past them (a job's A rows are read once per S block)
        std::vector<long long> bbase(n_jobs + 1);
        long long nbk = 0;
        for (int j = 0; j < n_jobs; ++j) {
            bbase[j] = nbk;
            const long long nsb = std::max<long long>(1, (nB[j] + b->sblock_rows - 1) / b->sblock_rows);
            nbk += (long long)nA[j] * nsb;
        }
        bbase[n_jobs] = nbk;
        b->n_buckets = nbk;
        if (nbk > 0 && nbk < 0xffffffffll) {
            if ((e = upload(b->bbase, bbase)) || (e = ensure(b->sorted, b->cand_cap * sizeof(uint2))) ||
                (e = ensure(b->sbuf, rescore_stream_batch_buf_bytes(nbk, sumA))))
                return fail(from_cuda(e));
            b->stream = true;
        }
    }

    if (flags & EJOIN_BATCH_AUTOTUNE) {
        if ((st = autotune(b)) != EJOIN_OK) return fail(st);
    }
    // one eager run with events between the stages: the stage split reported by ejoin_batch_info
    if (c->events) {
        if ((e = enqueue(b, c->stream, b->group_m, false, c->ev)) != cudaSuccess) return fail(from_cuda(e));
        if ((st = read_misc(b, hm, c->stream)) != EJOIN_OK) return fail(st);
        cudaEventElapsedTime(&b->ms_normalize, c->ev[0], c->ev[1]);
        cudaEventElapsedTime(&b->ms_contract, c->ev[1], c->ev[2]);
        cudaEventElapsedTime(&b->ms_rescore, c->ev[2], c->ev[3]);
    }
    if (flags & EJOIN_BATCH_GRAPH) {
        if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return fail(from_cuda(e));
        if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return fail(from_cuda(e));
        cudaError_t e2 = enqueue(b, b->cap_stream, b->group_m);
        cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, &b->graph);
        if (e2 != cudaSuccess || e3 != cudaSuccess) return fail(from_cuda(e2 != cudaSuccess ? e2 : e3));
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return fail(from_cuda(e));
    }
    // two normalisations, the contraction and the re-score (streaming path: row-to-job table, histogram,
    // three scan phases, scatter and the re-score); selections: count, scan and scatter per side, job table
    b->launches_per_run = (b->stream ? 10 : 4) + (has_sel ? 7 : 0);
    *out = b;
    return EJOIN_OK;
}

ejoin_status ejoin_batch_run(ejoin_batch *b)
{
    if (!b) return EJOIN_EINVAL;
    DeviceGuard g(b->ctx->device);
    cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, b->ctx->stream) : enqueue(b, b->ctx->stream, b->group_m);
    return from_cuda(e);
}

ejoin_status ejoin_batch_wait(ejoin_batch *b, uint64_t *count)
{
    if (!b || !count) return EJOIN_EINVAL;
    DeviceGuard g(b->ctx->device);
    DevMisc hm;
    ejoin_status st = read_misc(b, hm, b->ctx->stream);
    *count = hm.pair_count;
    if (st != EJOIN_OK) return st;
    if (hm.cand_count > b->cand_cap || hm.pair_count > b->pair_cap) return EJOIN_EOVERFLOW;
    b->ctx->stats = ejoin_stats{};
    b->ctx->stats.candidates = hm.cand_count;
    b->ctx->stats.pairs = hm.pair_count;
    b->ctx->stats.fp64_rescored = hm.band_count;
    b->ctx->stats.launches = b->launches_per_run;
    b->ctx->stats.band = b->band;
    return EJOIN_OK;
}

ejoin_status ejoin_batch_result(const ejoin_batch *b, const ejoin_batch_pair **d_pairs, uint64_t *capacity)
{
    if (!b || !d_pairs) return EJOIN_EINVAL;
    *d_pairs = (const ejoin_batch_pair *)b->pairs.p;
    if (capacity) *capacity = b->pair_cap;
    return EJOIN_OK;
}

ejoin_status ejoin_batch_info(const ejoin_batch *b, ejoin_batch_stats *out)
{
    if (!b || !out) return EJOIN_EINVAL;
    out->n_jobs = b->n_jobs;
    out->total_tiles = b->total_tiles;
    out->rows_r = b->rowsA;
    out->rows_s = b->rowsB;
    out->group_m = b->group_m;
    out->ms_normalize = b->ms_normalize;
    out->ms_contract = b->ms_contract;
    out->ms_rescore = b->ms_rescore;
    out->graph = b->exec != nullptr;
    out->candidate_capacity = b->cand_cap;
    out->pair_capacity = b->pair_cap;
    out->band = b->band;
    return EJOIN_OK;
}

void ejoin_batch_destroy(ejoin_batch *b) { destroy_batch(b); }

}  // extern "C"
