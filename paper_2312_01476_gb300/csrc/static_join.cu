// Allocation-free entry point: ejoin_threshold_static.
//
// Some callers cannot call cudaMalloc at all: a database executor or serving
// process whose device memory is owned by its own pool allocator, a process
// held to a fixed memory budget, or a latency-critical loop in which
// cudaMalloc / cudaFree would synchronise the device or fail under
// fragmentation.  For them this entry point runs the BF16 join (normalise,
// tcgen05 contraction with fused threshold, exact re-score) with all of its
// scratch in one file-scope device array of fixed size, so the call itself
// allocates nothing.  The caller passes the inputs and the output buffer.
//
// The array lives in this library's device image: every GPU that loads the
// library holds it (EJOIN_STATIC_SCRATCH_BYTES) until the process exits.  All
// calls share it and it keeps the contents of the last call, so the counters
// are cleared at the start of every call, and calls that overlap on the GPU
// (different streams, or different host threads on one device) race on it.
//
// The paper has no counterpart of this entry point.
#include <cudaTypedefs.h>

#include <mutex>

#include "host_internal.h"

using namespace ej;

namespace {

constexpr size_t MISC_BYTES = 1024;
constexpr size_t INV_BYTES = (size_t)EJOIN_STATIC_MAX_ROWS * 4;
constexpr size_t CAND_BYTES = (size_t)EJOIN_STATIC_MAX_CANDIDATES * 8;
constexpr size_t OPER_BYTES = (size_t)EJOIN_STATIC_MAX_OPERAND_ELEMS * 2;  // BF16
constexpr size_t OFF_MISC = 0;
constexpr size_t OFF_INV_A = OFF_MISC + MISC_BYTES;
constexpr size_t OFF_INV_B = OFF_INV_A + INV_BYTES;
constexpr size_t OFF_CAND = OFF_INV_B + INV_BYTES;
constexpr size_t OFF_BAND = OFF_CAND + CAND_BYTES;  // candidates near eps for the accurate tier
constexpr size_t OFF_OPER = OFF_BAND + CAND_BYTES;
constexpr size_t SCRATCH_BYTES = OFF_OPER + OPER_BYTES;
static_assert(SCRATCH_BYTES == EJOIN_STATIC_SCRATCH_BYTES, "scratch size stated in ejoin.h");
static_assert(OFF_OPER % 1024 == 0, "operand area alignment for TMA");
static_assert(sizeof(DevMisc) <= MISC_BYTES, "counter block");

// The scratch array.  Host code must not use its name as a device address:
// the address comes from cudaGetSymbolAddress in device_setup(), on every call.
static __device__ __align__(256) unsigned char g_static_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
// Per-device attributes that outlive any context (SM count, architecture).  The scratch array's address
// is not cached: a module can be reloaded into a new primary context (after cudaDeviceReset) at another
// address, so every call looks it up again with the device current.
struct DeviceInfo {
    bool ready = false;
    int num_sms = 0;
    bool sm103 = false;
};
DeviceInfo g_dev[MAX_DEVICES];
std::mutex g_mu;

ejoin_status device_setup(int dev, int *num_sms, bool *sm103, unsigned char **scratch)
{
    if (dev < 0 || dev >= MAX_DEVICES) return EJOIN_EUNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        DeviceInfo &s = g_dev[dev];
        if (!s.ready) {
            int sms = 0, major = 0, minor = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
                return EJOIN_ECUDA;
            s.num_sms = sms;
            s.sm103 = major == 10 && minor == 3;
            s.ready = true;
        }
        *num_sms = s.num_sms;
        *sm103 = s.sm103;
    }
    // `dev` is the current device here (the caller's)
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return EJOIN_ECUDA;
    *scratch = static_cast<unsigned char *>(p);
    return EJOIN_OK;
}

}  // namespace

extern "C" ejoin_status ejoin_threshold_static(ejoin_rel R, ejoin_rel S, float eps, ejoin_pair *d_pairs,
                                               uint64_t capacity, uint64_t *count, void *stream)
{
    if (!count) return EJOIN_EINVAL;
    *count = 0;
    if (R.d != S.d || R.d < 1 || R.d > 4096 || R.n < 0 || S.n < 0 || R.ld < R.d || S.ld < S.d) return EJOIN_EINVAL;
    if ((R.n && !R.x) || (S.n && !S.x) || (capacity && !d_pairs) || eps != eps) return EJOIN_EINVAL;
    // size limits of the fixed scratch array
    const int64_t kp = host::round_up(R.d, 64);
    const int64_t rowsA = host::round_up(R.n > 0 ? R.n : 1, 256), rowsB = host::round_up(S.n > 0 ? S.n : 1, 256);
    if (R.n > EJOIN_STATIC_MAX_ROWS || S.n > EJOIN_STATIC_MAX_ROWS ||
        (rowsA + rowsB) * kp > (int64_t)EJOIN_STATIC_MAX_OPERAND_ELEMS)
        return EJOIN_EINVAL;
    if (R.n == 0 || S.n == 0) return EJOIN_OK;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EJOIN_ECUDA;
    int num_sms = 0;
    bool sm103 = false;
    unsigned char *base = nullptr;
    ejoin_status st = device_setup(dev, &num_sms, &sm103, &base);
    if (st != EJOIN_OK) return st;
    if (!sm103) return EJOIN_EUNSUPPORTED;

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevMisc *dm = reinterpret_cast<DevMisc *>(base + OFF_MISC);
    float *invA = reinterpret_cast<float *>(base + OFF_INV_A);
    float *invB = reinterpret_cast<float *>(base + OFF_INV_B);
    uint2 *cand = reinterpret_cast<uint2 *>(base + OFF_CAND);
    uint2 *band_list = reinterpret_cast<uint2 *>(base + OFF_BAND);
    void *A = base + OFF_OPER;
    void *B = base + OFF_OPER + (size_t)rowsA * kp * 2;
    const float band = host::default_band(EJOIN_BF16, kp);  // the context path's rigorous default

    cudaError_t e;
    if ((e = cudaMemsetAsync(dm, 0, sizeof(DevMisc), s)) != cudaSuccess) return host::from_cuda(e);
    if ((e = launch_set_count(&dm->n_sel[0], R.n, s)) != cudaSuccess) return host::from_cuda(e);
    if ((e = launch_set_count(&dm->n_sel[1], S.n, s)) != cudaSuccess) return host::from_cuda(e);
    if ((e = launch_normalize(FMT_BF16, R.x, R.ld, R.d, nullptr, &dm->n_sel[0], R.n, A, kp, (int)kp, invA, nullptr,
                              &dm->status, num_sms, s)) != cudaSuccess)
        return host::from_cuda(e);
    if ((e = launch_normalize(FMT_BF16, S.x, S.ld, S.d, nullptr, &dm->n_sel[1], S.n, B, kp, (int)kp, invB, nullptr,
                              &dm->status, num_sms, s)) != cudaSuccess)
        return host::from_cuda(e);
    CUtensorMap tmA, tmB;
    if (!host::make_tmap(&tmA, A, FMT_BF16, kp, rowsA, 128) || !host::make_tmap(&tmB, B, FMT_BF16, kp, rowsB, 256))
        return EJOIN_ECUDA;
    if ((e = launch_sim_tc(0, &tmA, &tmB, (int)kp, &dm->n_sel[0], &dm->n_sel[1], eps - band, nullptr, nullptr, cand,
                           EJOIN_STATIC_MAX_CANDIDATES, &dm->cand_count, &dm->status, 1ull << 31, 0, num_sms,
                           default_group_m(kp), s)) != cudaSuccess)
        return host::from_cuda(e);
    if ((e = launch_rescore(cand, &dm->cand_count, EJOIN_STATIC_MAX_CANDIDATES, R.x, R.ld, S.x, S.ld, R.d, nullptr,
                            nullptr, invA, invB, eps, host::DEFAULT_FP64_BAND, d_pairs, capacity, &dm->pair_count,
                            &dm->band_count, 0, num_sms, s, band_list, EJOIN_STATIC_MAX_CANDIDATES)) != cudaSuccess)
        return host::from_cuda(e);
    DevMisc hm;
    if ((e = cudaMemcpyAsync(&hm, dm, sizeof(DevMisc), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return host::from_cuda(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return host::from_cuda(e);
    if (hm.status & ERR_NONFINITE) return EJOIN_ENONFINITE;
    if (hm.status & ERR_TIMEOUT) return EJOIN_ETIMEOUT;
    if (hm.status) return EJOIN_ECUDA;
    if (hm.cand_count > EJOIN_STATIC_MAX_CANDIDATES) return EJOIN_EOVERFLOW;  // *count stays 0: set incomplete
    *count = hm.pair_count;
    return hm.pair_count > capacity ? EJOIN_EOVERFLOW : EJOIN_OK;
}
