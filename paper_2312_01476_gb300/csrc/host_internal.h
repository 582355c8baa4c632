// Host-side internals shared by the C ABI translation units: the context,
// device buffers, tensor-map encoding, guard bands.
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "ejoin_internal.cuh"

namespace ej {
namespace host {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Grow-only device buffer (contents zeroed on growth).
cudaError_t ensure(Buf &b, size_t bytes);
void release(Buf &b);
ejoin_status from_cuda(cudaError_t e);
int fmt_of(int prec);
size_t fmt_bytes(int fmt);
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
// 2-D K-major operand [rows x kp] with a (128-byte x box_rows) box and 128-byte swizzle.
bool make_tmap(CUtensorMap *m, const void *base, int fmt, int64_t kp, int64_t rows, uint32_t box_rows);
// 2-D tensor map over raw FP32 rows (d columns, ld floats apart, columns past d read as zeros), a
// (32-float x box_rows) box, 128-byte swizzle; needs a 16-byte aligned base and ld % 4 == 0.
bool make_tmap_rows_f32(CUtensorMap *m, const float *base, int64_t d, int64_t ld, int64_t rows, uint32_t box_rows);
// Rigorous default guard band of a precision at padded dimension kp.
float default_band(int prec, int64_t kp);
// Default half-width around eps inside which the accurate tier (compensated dot products finished in
// FP64) decides a candidate instead of the FP32 re-score.
constexpr float DEFAULT_FP64_BAND = 2e-5f;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct Side {
    Buf norm, inv, scale, ids, blk_counts, blk_offsets;
};

constexpr int N_EV = 8;

}  // namespace host
}  // namespace ej

struct ejoin_ctx;
namespace ej {
namespace host {
// EJOIN_FLAG_SORT: sort the n records at `pairs` (device-accessible) by (i, j), i < n_i, j < n_j, on the
// context's stream, and synchronise.
ejoin_status sort_result(ejoin_ctx *c, ejoin_pair *pairs, uint64_t n, uint64_t n_i, uint64_t n_j);
// The accurate tier's per-row workspace for R.n and S.n rows (grown in the context).
cudaError_t band_norms(ejoin_ctx *c, int64_t nR, int64_t nS, BandNorms *bn);
}  // namespace host
}  // namespace ej

struct ejoin_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int prec = EJOIN_BF16;
    float band_cfg = -1.f;
    float fp64_band = 2e-5f;
    uint64_t cap_hint = 1u << 20;
    uint32_t flags = 0;
    uint64_t timeout = 1ull << 31;
    int group_m = 0;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    ej::host::Side side[2];
    ej::host::Buf misc;
    ej::host::Buf cand;
    uint64_t cand_cap = 0;
    ej::host::Buf band;  // candidates near eps for the accurate tier (as many slots as candidates)
    ej::host::Buf psorted;  // panel-ordered re-score: the candidates bucketed by panel of R rows
    ej::host::Buf pbuf;     // panel-ordered re-score: per-panel counts, offsets and chunk offsets
    ej::host::Buf sort_tmp, sort_scratch;  // EJOIN_FLAG_SORT: second record buffer and digit counts
    ej::host::Buf band_rows;               // accurate tier: per-row flags and squared norms of R and S
    ej::host::Buf top;     // top-k: per operand row scratch (maxima, thresholds, counts, offsets)
    ej::host::Buf topseg;  // top-k, k > 1: the candidates' keys bucketed by row
    ej::host::Buf host_in[6];
    ej::host::Buf host_pairs;
    cudaEvent_t ev[ej::host::N_EV] = {};
    bool events = false;
    ejoin_stats stats{};
};
