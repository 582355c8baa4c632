// C ABI of libejoin: context, workspace, argument validation, dispatch of the
// select -> normalise -> contract -> re-score pipeline, tensor-map encoding,
// and error reporting.  All device work goes through the kernels of this
// library; there is no host fallback.
//
// The pipeline evaluates the E-theta-join of Sec. III-C (Eq. (E-theta-Join))
// with the relational predicates pushed below the vector work (Eq.
// (E-Selection), Sec. VI-E pre-filter), in the tensor formulation of Sec.
// IV-C, tile by tile (Sec. V-B), mapping passing entries back to tuple ids
// through the partition offsets (Sec. IV-C).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "host_internal.h"

using namespace ej;

namespace ej {
namespace host {

cudaError_t ensure(Buf &b, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (b.bytes >= bytes) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) {
        b.bytes = bytes;
        // padding rows of the operand buffers are read by the contraction
        // (and masked); give them defined contents once
        e = cudaMemset(b.p, 0, bytes);
    }
    return e;
}

void release(Buf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}


ejoin_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return EJOIN_OK;
    if (e == cudaErrorMemoryAllocation) return EJOIN_ENOMEM;
    return EJOIN_ECUDA;
}

int fmt_of(int prec)
{
    switch (prec) {
    case EJOIN_BF16: return FMT_BF16;
    case EJOIN_FP8_E4M3: return FMT_FP8;
    default: return FMT_F32;
    }
}

size_t fmt_bytes(int fmt) { return fmt == FMT_BF16 ? 2 : (fmt == FMT_FP8 ? 1 : 4); }


// The driver's tensor-map encoder, looked up once (a function-local static: initialised once even when
// several host threads make their first call together).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// 2-D K-major operand [rows x kp] with a (128-byte x box_rows) box and 128-byte swizzle.
bool make_tmap(CUtensorMap *m, const void *base, int fmt, int64_t kp, int64_t rows, uint32_t box_rows)
{
    auto enc = encode_fn();
    if (!enc) return false;
    CUtensorMapDataType dt = fmt == FMT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                             : fmt == FMT_FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const size_t eb = fmt_bytes(fmt);
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(kp * eb)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / eb), box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}



// FP32 rows of a caller's matrix read in place: d columns (the K extent; the box's columns past d read
// as zeros), `rows` rows ld floats apart, a (32-float x box_rows) box, 128-byte swizzle.  Needs a
// 16-byte aligned base and ld % 4 == 0.
bool make_tmap_rows_f32(CUtensorMap *m, const float *base, int64_t d, int64_t ld, int64_t rows, uint32_t box_rows)
{
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {32u, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

float default_band(int prec, int64_t kp)
{
    const double g = (double)kp * std::ldexp(1.0, -24);  // FP32 accumulation over kp terms
    const double small = 8.0 * std::ldexp(1.0, -24);     // FP32 normalisation of both rows
    double b;
    switch (prec) {
    case EJOIN_BF16: {
        const double u = std::ldexp(1.0, -8);
        b = 2 * u + u * u + 2 * g + small;
        break;
    }
    case EJOIN_TF32: {
        const double u = std::ldexp(1.0, -10);  // conservative: truncation to 10 stored bits
        b = 2 * u + u * u + 2 * g + small;
        break;
    }
    case EJOIN_FP8_E4M3: {
        const double u = std::ldexp(1.0, -4);
        const double er = u + std::ldexp(1.0, -10) / 448.0 * std::sqrt((double)kp);
        b = 2 * er + er * er + 2 * g + small;
        break;
    }
    default: b = 2 * g + small; break;
    }
    return (float)(1.25 * b);
}

}  // namespace host
}  // namespace ej

using namespace ej::host;

namespace ej {
namespace host {
cudaError_t band_norms(ejoin_ctx *c, int64_t nR, int64_t nS, BandNorms *bn)
{
    nR = std::max<int64_t>(nR, 1);
    nS = std::max<int64_t>(nS, 1);
    const size_t bytes = (size_t)(nR + nS) * 12;
    cudaError_t e = ensure(c->band_rows, bytes);
    if (e != cudaSuccess) return e;
    char *p = (char *)c->band_rows.p;
    bn->nrmR = (double *)p;
    bn->nrmS = bn->nrmR + nR;
    bn->claimR = (unsigned *)(bn->nrmS + nS);
    bn->claimS = bn->claimR + nR;
    bn->nR = nR;
    bn->nS = nS;
    return cudaSuccess;
}

ejoin_status sort_result(ejoin_ctx *c, ejoin_pair *pairs, uint64_t n, uint64_t n_i, uint64_t n_j)
{
    if (n <= 1) return EJOIN_OK;
    if (n > 0xffffffffull) return EJOIN_EUNSUPPORTED;
    cudaError_t e;
    if ((e = ensure(c->sort_tmp, n * sizeof(ejoin_pair))) != cudaSuccess) return from_cuda(e);
    if ((e = ensure(c->sort_scratch, sort_pairs_scratch_bytes(n))) != cudaSuccess) return from_cuda(e);
    if ((e = launch_sort_pairs(pairs, (ejoin_pair *)c->sort_tmp.p, n, n_i, n_j, c->sort_scratch.p, c->stream)) !=
        cudaSuccess)
        return from_cuda(e);
    c->stats.launches += 1;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return from_cuda(e);
    return EJOIN_OK;
}
}  // namespace host
}  // namespace ej

extern "C" {

const char *ejoin_version(void) { return "ejoin-gb300 0.1 (sm_103a)"; }

const char *ejoin_strerror(ejoin_status s)
{
    switch (s) {
    case EJOIN_OK: return "ok";
    case EJOIN_EINVAL: return "invalid argument";
    case EJOIN_ENOMEM: return "device allocation failed";
    case EJOIN_EOVERFLOW: return "result exceeds the pair buffer capacity";
    case EJOIN_ENONFINITE: return "input holds NaN or Inf";
    case EJOIN_ECUDA: return "CUDA error";
    case EJOIN_ETIMEOUT: return "device-side wait timed out";
    case EJOIN_EUNSUPPORTED: return "unsupported precision or shape on this device";
    }
    return "unknown status";
}

int64_t ejoin_padded_dim(int32_t prec, int32_t d)
{
    if (d <= 0) return 0;
    switch (prec) {
    case EJOIN_BF16: return round_up(d, 64);
    case EJOIN_FP8_E4M3: return round_up(d, 128);
    case EJOIN_TF32: return round_up(d, 32);
    default: return round_up(d, 32);
    }
}

ejoin_status ejoin_create(ejoin_ctx **out, const ejoin_config *cfg)
{
    if (!out) return EJOIN_EINVAL;
    *out = nullptr;
    ejoin_ctx *c = new (std::nothrow) ejoin_ctx();
    if (!c) return EJOIN_ENOMEM;
    if (cfg) {
        c->device = cfg->device;
        c->stream = reinterpret_cast<cudaStream_t>(cfg->stream);
        c->prec = cfg->prec;
        c->band_cfg = cfg->band;
        c->fp64_band = cfg->fp64_band < 0.f ? DEFAULT_FP64_BAND : cfg->fp64_band;
        c->cap_hint = cfg->capacity_hint ? cfg->capacity_hint : (1u << 20);
        c->flags = cfg->flags;
        c->timeout = cfg->timeout_cycles ? cfg->timeout_cycles : (1ull << 31);
        c->group_m = cfg->group_m;
    }
    if (c->prec < EJOIN_F32 || c->prec > EJOIN_TF32) {
        delete c;
        return EJOIN_EINVAL;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || c->device < 0 || c->device >= ndev) {
        delete c;
        return e != cudaSuccess ? EJOIN_ECUDA : EJOIN_EINVAL;
    }
    DeviceGuard g(c->device);
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, c->device);
    if (e != cudaSuccess) {
        delete c;
        return EJOIN_ECUDA;
    }
    c->num_sms = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    if (c->prec != EJOIN_F32 && !(prop.major == 10 && prop.minor == 3)) {
        // the tensor-core kernels are built for sm_103a only
        delete c;
        return EJOIN_EUNSUPPORTED;
    }
    for (int i = 0; i < N_EV; ++i) {
        if (cudaEventCreate(&c->ev[i]) != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(c->ev[k]);
            delete c;
            return EJOIN_ECUDA;
        }
    }
    c->events = true;
    e = ensure(c->misc, sizeof(DevMisc));
    if (e != cudaSuccess) {
        ejoin_destroy(c);
        return from_cuda(e);
    }
    *out = c;
    return EJOIN_OK;
}

void ejoin_destroy(ejoin_ctx *c)
{
    if (!c) return;
    {
        DeviceGuard g(c->device);
        cudaStreamSynchronize(c->stream);
        for (auto &s : c->side) {
            release(s.norm);
            release(s.inv);
            release(s.scale);
            release(s.ids);
            release(s.blk_counts);
            release(s.blk_offsets);
        }
        release(c->misc);
        release(c->cand);
        release(c->band);
        release(c->psorted);
        release(c->pbuf);
        release(c->sort_tmp);
        release(c->sort_scratch);
        release(c->band_rows);
        release(c->top);
        release(c->topseg);
        for (auto &b : c->host_in) release(b);
        release(c->host_pairs);
        if (c->events)
            for (auto &ev : c->ev) cudaEventDestroy(ev);
    }
    delete c;
}

ejoin_status ejoin_set_timeout(ejoin_ctx *c, uint64_t timeout_cycles)
{
    if (!c) return EJOIN_EINVAL;
    c->timeout = timeout_cycles ? timeout_cycles : (1ull << 31);
    return EJOIN_OK;
}

ejoin_status ejoin_last_stats(const ejoin_ctx *c, ejoin_stats *out)
{
    if (!c || !out) return EJOIN_EINVAL;
    *out = c->stats;
    return EJOIN_OK;
}

ejoin_status ejoin_pairs_free(ejoin_ctx *c, ejoin_pairs *p)
{
    if (!c || !p) return EJOIN_EINVAL;
    if (p->d_pairs) {
        DeviceGuard g(c->device);
        cudaStreamSynchronize(c->stream);
        cudaFree(p->d_pairs);
    }
    p->d_pairs = nullptr;
    p->capacity = 0;
    return EJOIN_OK;
}

}  // extern "C"

namespace {

bool rel_ok(const ejoin_rel &r)
{
    if (r.n < 0 || r.n > (int64_t)0x7FFFFEFF) return false;
    if (r.d < 1 || r.d > 4096) return false;
    if (r.ld < r.d) return false;
    if (r.n > 0 && !r.x) return false;
    return true;
}

bool sel_ok(const ejoin_sel *s)
{
    if (!s) return true;
    if (!s->attr && !s->bits) return false;
    if (s->attr && (s->op < EJOIN_LT || s->op > EJOIN_NE)) return false;
    return true;
}

bool same_sel(const ejoin_sel *a, const ejoin_sel *b)
{
    if (!a || !b) return a == b;
    return a->attr == b->attr && a->bits == b->bits && (a->attr == nullptr || (a->op == b->op && a->c == b->c));
}


// Selection + normalisation of one relation into side buffers (or caller buffers).
ejoin_status prepare_side(ejoin_ctx *c, int which, const ejoin_rel &r, const ejoin_sel *sel, int fmt, int64_t kp,
                          void *out, int64_t ld_out, float *inv, float *scale, uint32_t *ids, long long *n_sel,
                          unsigned *status, bool timing_split, int scale_group = 0, float *raw_out = nullptr,
                          int64_t raw_ld = 0)
{
    Side &sd = c->side[which];
    cudaError_t e;
    if (sel) {
        const int64_t nb = std::max<int64_t>(1, (r.n + SEL_ROWS_PER_BLOCK - 1) / SEL_ROWS_PER_BLOCK);
        if ((e = ensure(sd.blk_counts, nb * 4)) != cudaSuccess) return from_cuda(e);
        if ((e = ensure(sd.blk_offsets, nb * 4)) != cudaSuccess) return from_cuda(e);
        SelArgs s{sel->attr, sel->op, sel->c, sel->bits};
        uint32_t *bc = (uint32_t *)sd.blk_counts.p, *bo = (uint32_t *)sd.blk_offsets.p;
        if ((e = launch_sel_count(s, r.n, bc, c->stream)) != cudaSuccess) return from_cuda(e);
        if ((e = launch_sel_scan(bc, (r.n + SEL_ROWS_PER_BLOCK - 1) / SEL_ROWS_PER_BLOCK, bo, n_sel, c->stream)) !=
            cudaSuccess)
            return from_cuda(e);
        if ((e = launch_sel_scatter(s, r.n, bo, ids, c->stream)) != cudaSuccess) return from_cuda(e);
        c->stats.launches += r.n > 0 ? 3 : 1;
    } else {
        if ((e = launch_set_count(n_sel, (long long)r.n, c->stream)) != cudaSuccess) return from_cuda(e);
        c->stats.launches += 1;
    }
    if (timing_split && (c->flags & EJOIN_FLAG_TIMING)) cudaEventRecord(c->ev[1 + which], c->stream);
    if (r.n > 0) {
        if (fmt == FMT_FP8 && scale_group > 0) {
            e = launch_normalize_fp8_grouped(r.x, r.ld, r.d, sel ? ids : nullptr, n_sel, r.n, out, ld_out, (int)kp, inv,
                                             scale, scale_group, status, c->num_sms, c->stream, raw_out, raw_ld);
            c->stats.launches += 3;
        } else {
            e = launch_normalize(fmt, r.x, r.ld, r.d, sel ? ids : nullptr, n_sel, r.n, out, ld_out, (int)kp, inv,
                                 scale, status, c->num_sms, c->stream, raw_out, raw_ld);
            c->stats.launches += 1;
        }
        if (e != cudaSuccess) return from_cuda(e);
    }
    return EJOIN_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.f;
    return ms;
}

// The device error word as a status: non-finite input first, then an expired wait, then anything else.
ejoin_status status_of(unsigned err)
{
    if (err & ERR_NONFINITE) return EJOIN_ENONFINITE;
    if (err & ERR_TIMEOUT) return EJOIN_ETIMEOUT;
    return err ? EJOIN_ECUDA : EJOIN_OK;
}

// Workspace of one operand side: n rows (rounded up to whole 256-row tiles) of kp elements in format fmt,
// their inverse norms, e4m3 scales, and the kept-row ids when a selection is given.
cudaError_t ensure_operand(Side &sd, int64_t n, int64_t kp, int fmt, bool with_ids)
{
    const int64_t rows = round_up(std::max<int64_t>(n, 1), 256);
    cudaError_t e;
    if ((e = ensure(sd.norm, (size_t)rows * kp * fmt_bytes(fmt))) != cudaSuccess) return e;
    if ((e = ensure(sd.inv, (size_t)rows * 4)) != cudaSuccess) return e;
    if (fmt == FMT_FP8 && (e = ensure(sd.scale, (size_t)rows * 4)) != cudaSuccess) return e;
    if (with_ids && (e = ensure(sd.ids, (size_t)rows * 4)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Device pipeline shared by ejoin_threshold and ejoin_threshold_host.
// rawR / rawS (optional): device buffers of R.n x R.d / S.n x S.d floats.  R and S are then read only by the
// normalisation pass (they may sit in device-accessible host memory), which copies each kept row there at
// its row number; the re-score reads those copies.
ejoin_status run_threshold(ejoin_ctx *c, const ejoin_rel &R, const ejoin_rel &S, float eps, const ejoin_sel *selR,
                           const ejoin_sel *selS, ejoin_pair **pairs_io, uint64_t *cap_io, bool may_alloc,
                           uint64_t *d_count_user, uint64_t *count_out, float *rawR = nullptr, float *rawS = nullptr)
{
    c->stats = ejoin_stats{};
    if (!rel_ok(R) || !rel_ok(S) || R.d != S.d || !sel_ok(selR) || !sel_ok(selS)) return EJOIN_EINVAL;
    if (std::isnan(eps)) return EJOIN_EINVAL;
    const bool timing = (c->flags & EJOIN_FLAG_TIMING) != 0;
    const bool count_only = (c->flags & EJOIN_FLAG_COUNT_ONLY) != 0;
    const int prec = c->prec;
    const int fmt = fmt_of(prec);
    const int64_t kp = ejoin_padded_dim(prec, R.d);
    const bool self = R.x == S.x && R.n == S.n && R.ld == S.ld && same_sel(selR, selS);
    const float band = c->band_cfg >= 0.f ? c->band_cfg : default_band(prec, kp);
    c->stats.band = band;
    cudaError_t e;

    // workspace
    const ejoin_rel *rels[2] = {&R, &S};
    const ejoin_sel *sels[2] = {selR, selS};
    for (int w = 0; w < (self ? 1 : 2); ++w)
        if ((e = ensure_operand(c->side[w], rels[w]->n, kp, fmt, sels[w] != nullptr)) != cudaSuccess)
            return from_cuda(e);
    if (c->cand_cap == 0) c->cand_cap = c->cap_hint;
    if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
    DevMisc *dm = (DevMisc *)c->misc.p;
    if ((e = cudaMemsetAsync(dm, 0, sizeof(DevMisc), c->stream)) != cudaSuccess) return from_cuda(e);

    if (timing) cudaEventRecord(c->ev[0], c->stream);
    Side &sa = c->side[0];
    Side &sb = self ? c->side[0] : c->side[1];
    // e4m3: the S operand's scales are shared per 256-row column tile (a self-join's single operand too),
    // so the contraction folds them into its threshold; R keeps per-row scales
    ejoin_status st = prepare_side(c, 0, R, selR, fmt, kp, sa.norm.p, kp, (float *)sa.inv.p, (float *)sa.scale.p,
                                   (uint32_t *)sa.ids.p, &dm->n_sel[0], &dm->status, false, self ? 256 : 0, rawR,
                                   R.d);
    if (st != EJOIN_OK) return st;
    if (!self) {
        st = prepare_side(c, 1, S, selS, fmt, kp, sb.norm.p, kp, (float *)sb.inv.p, (float *)sb.scale.p,
                          (uint32_t *)sb.ids.p, &dm->n_sel[1], &dm->status, false, 256, rawS, S.d);
        if (st != EJOIN_OK) return st;
    }
    const long long *nA = &dm->n_sel[0];
    const long long *nB = self ? &dm->n_sel[0] : &dm->n_sel[1];
    if (timing) cudaEventRecord(c->ev[1], c->stream);
    // the rows the re-score gathers: the device copies when given, else R and S themselves
    const float *xR = rawR ? rawR : R.x, *xS = rawS ? rawS : (self && rawR ? rawR : S.x);
    const int64_t ldR = rawR ? R.d : R.ld, ldS = rawS ? S.d : (self && rawR ? R.d : S.ld);

    // bulk contraction -> candidates
    const float thr = eps - band;
    CUtensorMap tmA, tmB;
    if (prec != EJOIN_F32) {
        const int64_t rowsA = round_up(std::max<int64_t>(R.n, 1), 256);
        const int64_t rowsB = round_up(std::max<int64_t>(S.n, 1), 256);
        if (!make_tmap(&tmA, sa.norm.p, fmt, kp, rowsA, 128) || !make_tmap(&tmB, sb.norm.p, fmt, kp, rowsB, 256))
            return EJOIN_ECUDA;
    }
    const bool aligned_rows = R.d % 4 == 0 && ldR % 4 == 0 && ldS % 4 == 0 &&
                              (reinterpret_cast<uintptr_t>(xR) & 15) == 0 && (reinterpret_cast<uintptr_t>(xS) & 15) == 0;
    const bool fuse = prec != EJOIN_F32 && (c->flags & EJOIN_FLAG_FUSED) && aligned_rows &&
                      (*pairs_io != nullptr || count_only);
    if (fuse) {
        // contraction with the exact re-score fused in: one launch writes the final pairs
        FuseArgs fa{};
        fa.R = xR;
        fa.ldR = ldR;
        fa.S = xS;
        fa.ldS = ldS;
        fa.d = R.d;
        fa.idsR = selR ? (const uint32_t *)sa.ids.p : nullptr;
        fa.idsS = selS ? (const uint32_t *)sb.ids.p : nullptr;
        fa.invR = (const float *)sa.inv.p;
        fa.invS = (const float *)sb.inv.p;
        fa.eps = eps;
        fa.fp64_band = c->fp64_band;
        fa.out = *pairs_io;
        fa.out_cap = count_only ? 0 : *cap_io;
        fa.pair_count = &dm->pair_count;
        fa.band_count = &dm->band_count;
        fa.count_only = count_only ? 1 : 0;
        const int kind = prec == EJOIN_BF16 ? 0 : (prec == EJOIN_FP8_E4M3 ? 1 : 2);
        e = launch_sim_tc_fused(kind, &tmA, &tmB, (int)kp, nA, nB, thr, (const float *)sa.scale.p,
                                (const float *)sb.scale.p, fa, &dm->cand_count, &dm->status, c->timeout, c->num_sms,
                                c->group_m > 0 ? c->group_m : default_group_m(kp), c->stream);
        if (e != cudaSuccess) return from_cuda(e);
        c->stats.launches += 1;
        c->stats.fused = 1;
        if (timing) cudaEventRecord(c->ev[2], c->stream);
        if (d_count_user &&
            (e = cudaMemcpyAsync(d_count_user, &dm->pair_count, sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                 c->stream)) != cudaSuccess)
            return from_cuda(e);
        DevMisc hf;
        if ((e = cudaMemcpyAsync(&hf, dm, sizeof(DevMisc), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return from_cuda(e);
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return from_cuda(e);
        c->stats.n_sel_r = (uint64_t)hf.n_sel[0];
        c->stats.n_sel_s = (uint64_t)(self ? hf.n_sel[0] : hf.n_sel[1]);
        if (hf.status) return status_of(hf.status);
        c->stats.candidates = hf.cand_count;
        c->stats.pairs = hf.pair_count;
        c->stats.fp64_rescored = hf.band_count;
        if (timing) {
            c->stats.ms_normalize = elapsed(c->ev[0], c->ev[1]);
            c->stats.ms_contract = elapsed(c->ev[1], c->ev[2]);
            c->stats.ms_rescore = 0.f;
            c->stats.ms_total = elapsed(c->ev[0], c->ev[2]);
        }
        *count_out = hf.pair_count;
        if (!count_only && hf.pair_count > *cap_io) return EJOIN_EOVERFLOW;
        if ((c->flags & EJOIN_FLAG_SORT) && !count_only) return sort_result(c, *pairs_io, hf.pair_count, R.n, S.n);
        return EJOIN_OK;
    }
    // a self-join on the tensor cores contracts the upper triangle only (mirrored in the re-score)
    const bool sym = self && prec != EJOIN_F32 && !(c->flags & EJOIN_FLAG_NO_SYMMETRY);
    auto contract = [&]() -> ejoin_status {
        cudaError_t ee;
        if (sym) {
            const int kind = prec == EJOIN_BF16 ? 0 : (prec == EJOIN_FP8_E4M3 ? 1 : 2);
            ee = launch_sim_tc_sym(kind, &tmA, &tmB, (int)kp, nA, thr, (const float *)sa.scale.p, (uint2 *)c->cand.p,
                                   c->cand_cap, &dm->cand_count, &dm->status, c->timeout, 0, c->num_sms,
                                   c->group_m > 0 ? c->group_m : default_group_m(kp), c->stream);
        } else if (prec == EJOIN_F32) {
            ee = launch_sim_simt((const float *)sa.norm.p, (const float *)sb.norm.p, (int)kp, nA, nB, thr,
                                 (uint2 *)c->cand.p, c->cand_cap, &dm->cand_count, 0, c->num_sms, c->stream);
        } else {
            const int kind = prec == EJOIN_BF16 ? 0 : (prec == EJOIN_FP8_E4M3 ? 1 : 2);
            ee = launch_sim_tc(kind, &tmA, &tmB, (int)kp, nA, nB, thr, (const float *)sa.scale.p,
                               (const float *)sb.scale.p, (uint2 *)c->cand.p, c->cand_cap, &dm->cand_count,
                               &dm->status, c->timeout, 0, c->num_sms,
                               c->group_m > 0 ? c->group_m : default_group_m(kp), c->stream);
        }
        c->stats.launches += 1;
        return from_cuda(ee);
    };
    if ((st = contract()) != EJOIN_OK) return st;
    if (timing) cudaEventRecord(c->ev[2], c->stream);

    DevMisc hm;
    auto read_misc = [&]() -> cudaError_t {
        cudaError_t ee = cudaMemcpyAsync(&hm, dm, sizeof(DevMisc), cudaMemcpyDeviceToHost, c->stream);
        return ee == cudaSuccess ? cudaStreamSynchronize(c->stream) : ee;
    };
    // exact re-score of the candidates (it reads their count on the device): panel-ordered where the rows
    // allow it (R rows staged in shared memory per panel), else plain gathers in emission order.  Joins of
    // fewer than PANEL_MIN_PAIRS pairs (before selection) keep the gathers: their few candidates do not repay
    // the bucket sort, and the call then needs a single synchronisation.
    constexpr double PANEL_MIN_PAIRS = 134217728.0;  // 2^27
    const bool panels = aligned_rows && R.d <= 1024 && !(c->flags & EJOIN_FLAG_GATHER_RESCORE) &&
                        ((c->flags & EJOIN_FLAG_PANEL_RESCORE) || (double)R.n * (double)S.n >= PANEL_MIN_PAIRS);
    auto rescore = [&]() -> cudaError_t {
        cudaError_t ee = ensure(c->band, c->cand_cap * sizeof(uint2));
        if (ee != cudaSuccess) return ee;
        BandNorms bn;
        if (c->fp64_band > 0.f && (ee = band_norms(c, R.n, S.n, &bn)) != cudaSuccess) return ee;
        const BandNorms *bnp = c->fp64_band > 0.f ? &bn : nullptr;
        const uint32_t *idsA = selR ? (const uint32_t *)sa.ids.p : nullptr;
        const uint32_t *idsB = selS ? (const uint32_t *)sb.ids.p : nullptr;
        if (panels) {
            // the kept rows and the candidates are known here (read back before the re-score): they size the
            // panels and decide how far S blocks may split them
            const int64_t rows_a = std::max<long long>(hm.n_sel[0], 1);
            const int64_t rows_b = std::max<long long>(self ? hm.n_sel[0] : hm.n_sel[1], 1);
            const uint64_t hint = std::max<unsigned long long>(hm.cand_count, 1);
            if ((ee = ensure(c->psorted, c->cand_cap * sizeof(uint2))) != cudaSuccess) return ee;
            if ((ee = ensure(c->pbuf, rescore_panel_buf_bytes(rows_a, rows_b, R.d, hint))) != cudaSuccess) return ee;
            ee = launch_rescore_panels((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, (uint2 *)c->psorted.p,
                                       c->pbuf.p, rows_a, rows_b, hint, nA, xR, ldR, xS, ldS, R.d, idsA, idsB,
                                       (const float *)sa.inv.p,
                                       (const float *)sb.inv.p, eps, c->fp64_band, *pairs_io,
                                       count_only ? 0 : *cap_io, &dm->pair_count, &dm->band_count,
                                       count_only ? 1 : 0, c->num_sms, c->stream, (uint2 *)c->band.p, c->cand_cap,
                                       sym ? 1 : 0, bnp);
            if (ee != cudaSuccess) return ee;
            c->stats.launches += c->fp64_band > 0.f ? 10 : 6;
        } else {
            ee = launch_rescore((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, xR, ldR, xS, ldS, R.d, idsA,
                                idsB, (const float *)sa.inv.p, (const float *)sb.inv.p, eps, c->fp64_band, *pairs_io,
                                count_only ? 0 : *cap_io, &dm->pair_count, &dm->band_count, count_only ? 1 : 0,
                                c->num_sms, c->stream, (uint2 *)c->band.p, c->cand_cap, sym ? 1 : 0, bnp);
            if (ee != cudaSuccess) return ee;
            c->stats.launches += c->fp64_band > 0.f ? 5 : 1;
        }
        if (timing) cudaEventRecord(c->ev[3], c->stream);
        if (d_count_user)
            ee = cudaMemcpyAsync(d_count_user, &dm->pair_count, sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                 c->stream);
        return ee;
    };
    // With the result buffer known, the emission-order re-score is launched before the candidate count is
    // read back: one host synchronisation per call.  If the candidates overflowed their buffer, its pairs
    // are discarded and the call continues as below.  The panel-ordered re-score is sized by the counts,
    // so it follows their read-back.
    bool done = false;
    if ((*pairs_io != nullptr || count_only) && !panels) {
        if ((e = rescore()) != cudaSuccess) return from_cuda(e);
        if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
        if (hm.status) return status_of(hm.status);
        done = hm.cand_count <= c->cand_cap;
        if (!done) {
            if ((e = cudaMemsetAsync(&dm->pair_count, 0, 2 * sizeof(unsigned long long), c->stream)) != cudaSuccess)
                return from_cuda(e);
        }
    } else {
        if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
        if (hm.status) return status_of(hm.status);
    }
    if (!done) {
        while (hm.cand_count > c->cand_cap) {
            // candidate buffer too small: grow and run the contraction again
            c->cand_cap = hm.cand_count + hm.cand_count / 4 + 1024;
            if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
            if ((e = cudaMemsetAsync(&dm->cand_count, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess)
                return from_cuda(e);
            if ((st = contract()) != EJOIN_OK) return st;
            if (timing) cudaEventRecord(c->ev[2], c->stream);
            if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
            if (hm.status) return status_of(hm.status);
            c->stats.contract_retries++;
        }
        // result buffer
        if (*pairs_io == nullptr && may_alloc && !count_only) {
            // a symmetric self-join writes each off-diagonal candidate in both orders
            const uint64_t cap = std::max<uint64_t>(sym ? 2 * hm.cand_count : hm.cand_count, 1);
            void *p = nullptr;
            if ((e = cudaMalloc(&p, cap * sizeof(ejoin_pair))) != cudaSuccess) return from_cuda(e);
            *pairs_io = (ejoin_pair *)p;
            *cap_io = cap;
        }
        if (*pairs_io == nullptr && !count_only) *cap_io = 0;
        if ((e = rescore()) != cudaSuccess) return from_cuda(e);
        if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
        if (hm.status) return status_of(hm.status);
    }
    c->stats.n_sel_r = (uint64_t)hm.n_sel[0];
    c->stats.n_sel_s = (uint64_t)(self ? hm.n_sel[0] : hm.n_sel[1]);
    c->stats.candidates = hm.cand_count;
    c->stats.pairs = hm.pair_count;
    c->stats.fp64_rescored = hm.band_count;
    if (timing) {
        c->stats.ms_normalize = elapsed(c->ev[0], c->ev[1]);
        c->stats.ms_contract = elapsed(c->ev[1], c->ev[2]);
        c->stats.ms_rescore = elapsed(c->ev[2], c->ev[3]);
        c->stats.ms_total = elapsed(c->ev[0], c->ev[3]);
    }
    *count_out = hm.pair_count;
    if (!count_only && hm.pair_count > *cap_io) return EJOIN_EOVERFLOW;
    if ((c->flags & EJOIN_FLAG_SORT) && !count_only) return sort_result(c, *pairs_io, hm.pair_count, R.n, S.n);
    return EJOIN_OK;
}

// Top-k join condition (Sec. VI-E) on the tensor cores, 1 <= k <= 32.  k > 1 (and e4m3): pass 0 takes
// every R row's largest bulk similarity per column group, and the k-th largest group maximum, a lower
// bound of the row's k-th largest bulk similarity, becomes its threshold; pass 1 keeps the columns
// within 2 * band of the threshold: the bulk error is at most band, so they hold the exact top k.
// k = 1 otherwise: a single pass keeps the columns within 2 * band of the running row maximum.  The
// FP32 re-score then picks the best k of the candidates per row.
ejoin_status run_topk(ejoin_ctx *c, const ejoin_rel &R, const ejoin_rel &S, int k, const ejoin_sel *selR,
                      const ejoin_sel *selS, ejoin_pair **pairs_io, uint64_t *cap_io, bool may_alloc,
                      uint64_t *count_out)
{
    c->stats = ejoin_stats{};
    if (!rel_ok(R) || !rel_ok(S) || R.d != S.d || !sel_ok(selR) || !sel_ok(selS)) return EJOIN_EINVAL;
    if (k < 1 || k > TOPK_MAX_K) return EJOIN_EINVAL;
    const int prec = c->prec;
    if (prec == EJOIN_F32) return EJOIN_EUNSUPPORTED;
    const bool timing = (c->flags & EJOIN_FLAG_TIMING) != 0;
    const int fmt = fmt_of(prec);
    const int64_t kp = ejoin_padded_dim(prec, R.d);
    const bool self = R.x == S.x && R.n == S.n && R.ld == S.ld && same_sel(selR, selS);
    const float band = c->band_cfg >= 0.f ? c->band_cfg : default_band(prec, kp);
    c->stats.band = band;
    cudaError_t e;
    const ejoin_rel *rels[2] = {&R, &S};
    const ejoin_sel *sels[2] = {selR, selS};
    for (int w = 0; w < (self ? 1 : 2); ++w)
        if ((e = ensure_operand(c->side[w], rels[w]->n, kp, fmt, sels[w] != nullptr)) != cudaSuccess)
            return from_cuda(e);
    const int64_t rowsA = round_up(std::max<int64_t>(R.n, 1), 256);
    const int64_t rowsB = round_up(std::max<int64_t>(S.n, 1), 256);
    // k > 1, and e4m3 at any k (whose wide band makes the early running maximum of one pass a poor
    // threshold): a sampled first pass and a threshold kernel before the candidate pass
    const bool two_pass = k > 1 || fmt == FMT_FP8;
    // column groups of pass 0: 256 columns (one column tile), wider when the group maxima would
    // exceed TOPK_MAX_GROUPS per row or 4 GiB in all
    int shift = 62;
    int64_t ld = 1;
    if (two_pass) {
        const int64_t nS = std::max<int64_t>(S.n, 1);
        for (shift = 8;; ++shift) {
            ld = ((nS - 1) >> shift) + 1;
            if (ld <= TOPK_MAX_GROUPS && (double)rowsA * (double)ld * 4.0 <= 4294967296.0) break;
        }
    }
    // per-row scratch, zeroed: the best key (u64, k = 1); the threshold or running maximum, count,
    // offset and fill (u32 each); the group maxima of pass 0
    const size_t top_bytes = (size_t)rowsA * 24 + (two_pass ? (size_t)rowsA * ld * 4 : 0);
    if ((e = ensure(c->top, top_bytes)) != cudaSuccess) return from_cuda(e);
    unsigned long long *best = (unsigned long long *)c->top.p;
    unsigned *thr = (unsigned *)(best + rowsA);
    unsigned *row_cnt = thr + rowsA, *row_off = thr + 2 * rowsA, *row_fill = thr + 3 * rowsA;
    unsigned *gmax = thr + 4 * rowsA;
    if (c->cand_cap == 0) c->cand_cap = c->cap_hint;
    if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
    DevMisc *dm = (DevMisc *)c->misc.p;
    if ((e = cudaMemsetAsync(dm, 0, sizeof(DevMisc), c->stream)) != cudaSuccess) return from_cuda(e);
    if ((e = cudaMemsetAsync(c->top.p, 0, top_bytes, c->stream)) != cudaSuccess) return from_cuda(e);

    if (timing) cudaEventRecord(c->ev[0], c->stream);
    Side &sa = c->side[0];
    Side &sb = self ? c->side[0] : c->side[1];
    // e4m3: both operands' scales shared per 256-row tile (S's fold into the epilogue threshold)
    ejoin_status st = prepare_side(c, 0, R, selR, fmt, kp, sa.norm.p, kp, (float *)sa.inv.p, (float *)sa.scale.p,
                                   (uint32_t *)sa.ids.p, &dm->n_sel[0], &dm->status, false, self ? 256 : 0);
    if (st != EJOIN_OK) return st;
    if (!self) {
        st = prepare_side(c, 1, S, selS, fmt, kp, sb.norm.p, kp, (float *)sb.inv.p, (float *)sb.scale.p,
                          (uint32_t *)sb.ids.p, &dm->n_sel[1], &dm->status, false, 256);
        if (st != EJOIN_OK) return st;
    }
    const long long *nA = &dm->n_sel[0];
    const long long *nB = self ? &dm->n_sel[0] : &dm->n_sel[1];
    if (timing) cudaEventRecord(c->ev[1], c->stream);

    CUtensorMap tmA, tmB;
    if (!make_tmap(&tmA, sa.norm.p, fmt, kp, rowsA, 128) || !make_tmap(&tmB, sb.norm.p, fmt, kp, rowsB, 256))
        return EJOIN_ECUDA;
    const int kind = prec == EJOIN_BF16 ? 0 : (prec == EJOIN_FP8_E4M3 ? 1 : 2);
    const int gm = c->group_m > 0 ? c->group_m : default_group_m(kp);
    const float margin = 2.f * band;
    if (two_pass) {
        // pass 0 on every 8th column tile (at least 4k of them): the k-th largest maximum over any set
        // of column groups bounds the k-th largest similarity from below, the sample only loosens it
        e = launch_sim_tc_top(kind, 0, &tmA, &tmB, (int)kp, nA, nB, (const float *)sa.scale.p,
                              (const float *)sb.scale.p, gmax, ld, shift, TOPK_SAMPLE_STRIDE, 4 * k, margin,
                              (uint2 *)c->cand.p, c->cand_cap, &dm->cand_count, &dm->status, c->timeout, c->num_sms,
                              gm, c->stream);
        if (e == cudaSuccess) e = launch_topk_threshold(gmax, ld, shift, nA, rowsA, nB, k, thr, c->num_sms, c->stream);
        if (e != cudaSuccess) return from_cuda(e);
        c->stats.launches += 2;
    }
    // one pass (k = 1, not e4m3): on the running row maximum in thr (a repeat after a candidate overflow
    // starts from the final maxima and keeps only the columns within the margin of them)
    auto pass1 = [&]() -> cudaError_t {
        c->stats.launches += 1;
        return launch_sim_tc_top(kind, two_pass ? 1 : 2, &tmA, &tmB, (int)kp, nA, nB, (const float *)sa.scale.p,
                                 (const float *)sb.scale.p, thr, 1, 62, 1, 1, margin, (uint2 *)c->cand.p,
                                 c->cand_cap,
                                 &dm->cand_count, &dm->status, c->timeout, c->num_sms, gm, c->stream);
    };
    if ((e = pass1()) != cudaSuccess) return from_cuda(e);
    if (timing) cudaEventRecord(c->ev[2], c->stream);
    DevMisc hm;
    auto read_misc = [&]() -> cudaError_t {
        cudaError_t ee = cudaMemcpyAsync(&hm, dm, sizeof(DevMisc), cudaMemcpyDeviceToHost, c->stream);
        return ee == cudaSuccess ? cudaStreamSynchronize(c->stream) : ee;
    };
    if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
    c->stats.n_sel_r = (uint64_t)hm.n_sel[0];
    c->stats.n_sel_s = (uint64_t)(self ? hm.n_sel[0] : hm.n_sel[1]);
    if (hm.status) return status_of(hm.status);
    while (hm.cand_count > c->cand_cap) {
        // candidate buffer too small: grow it and run pass 1 again (the thresholds stay)
        c->cand_cap = hm.cand_count + hm.cand_count / 4 + 1024;
        if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
        if ((e = cudaMemsetAsync(&dm->cand_count, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess)
            return from_cuda(e);
        if ((e = pass1()) != cudaSuccess) return from_cuda(e);
        if (timing) cudaEventRecord(c->ev[2], c->stream);
        if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
        if (hm.status) return status_of(hm.status);
        c->stats.contract_retries++;
    }
    c->stats.candidates = hm.cand_count;
    if (k > 1 && hm.cand_count >= (1ull << 32)) return EJOIN_EUNSUPPORTED;  // 32-bit row offsets
    const uint64_t kk = std::min<uint64_t>((uint64_t)k, c->stats.n_sel_s);
    const uint64_t n_out = c->stats.n_sel_r * kk;
    if (*pairs_io == nullptr && may_alloc && n_out > 0) {
        void *p = nullptr;
        if ((e = cudaMalloc(&p, n_out * sizeof(ejoin_pair))) != cudaSuccess) return from_cuda(e);
        *pairs_io = (ejoin_pair *)p;
        *cap_io = n_out;
    }
    if (*pairs_io == nullptr) *cap_io = 0;
    const uint32_t *idsR = selR ? (const uint32_t *)sa.ids.p : nullptr;
    const uint32_t *idsS = selS ? (const uint32_t *)sb.ids.p : nullptr;
    if (hm.cand_count > 0 && k == 1) {
        e = launch_top1_rescore((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, R.x, R.ld, S.x, S.ld, R.d,
                                idsR, idsS, (const float *)sa.inv.p, (const float *)sb.inv.p, best, c->num_sms,
                                c->stream);
        if (e == cudaSuccess)
            e = launch_top1_emit(best, nA, rowsA, idsR, *pairs_io, *cap_io, &dm->pair_count, c->num_sms, c->stream);
        if (e != cudaSuccess) return from_cuda(e);
        c->stats.launches += 2;
    } else if (hm.cand_count > 0) {
        // keys beside the candidates, then bucketed by row
        if ((e = ensure(c->band, c->cand_cap * 8)) != cudaSuccess) return from_cuda(e);
        if ((e = ensure(c->topseg, c->cand_cap * 8)) != cudaSuccess) return from_cuda(e);
        unsigned long long *keys = (unsigned long long *)c->band.p, *seg = (unsigned long long *)c->topseg.p;
        e = launch_topk_rescore((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, R.x, R.ld, S.x, S.ld, R.d,
                                idsR, idsS, (const float *)sa.inv.p, (const float *)sb.inv.p, keys, row_cnt,
                                c->num_sms, c->stream);
        if (e == cudaSuccess) e = launch_sel_scan(row_cnt, rowsA, row_off, (long long *)&dm->pad2[0], c->stream);
        if (e == cudaSuccess)
            e = launch_topk_scatter((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, keys, row_off, row_fill,
                                    seg, c->num_sms, c->stream);
        if (e == cudaSuccess)
            e = launch_topk_select(seg, row_off, row_cnt, nA, rowsA, (int)kk, idsR, *pairs_io, *cap_io,
                                   &dm->pair_count, c->num_sms, c->stream);
        if (e != cudaSuccess) return from_cuda(e);
        c->stats.launches += 4;
    }
    if (timing) cudaEventRecord(c->ev[3], c->stream);
    if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
    if (hm.status) return status_of(hm.status);
    if (hm.pair_count) return EJOIN_ECUDA;  // a kept row with fewer candidates than records
    c->stats.pairs = n_out;
    if (timing) {
        c->stats.ms_normalize = elapsed(c->ev[0], c->ev[1]);
        c->stats.ms_contract = elapsed(c->ev[1], c->ev[2]);
        c->stats.ms_rescore = elapsed(c->ev[2], c->ev[3]);
        c->stats.ms_total = elapsed(c->ev[0], c->ev[3]);
    }
    *count_out = n_out;
    if (n_out > *cap_io) return EJOIN_EOVERFLOW;
    return EJOIN_OK;
}

// ℰ-selection (Sec. III-C, Eq. (ℰ-Selection)) of R against a batch of queries Q: the pairs (i, q) with
// selR(i) and cos(R_i, Q_q) >= eps.  Without a selection, and for rows that meet the TMA alignment, the
// scan reads R in place once (esel.cu); otherwise (or when a row's sum of squares leaves the FP32
// range) the kept rows are first compacted and normalised.  The candidates of every 64-query chunk
// go to one list, which the threshold join's re-score decides exactly.
ejoin_status run_eselect(ejoin_ctx *c, const ejoin_rel &R, const ejoin_sel *selR, const ejoin_rel &Q, float eps,
                         ejoin_pair **pairs_io, uint64_t *cap_io, bool may_alloc, uint64_t *count_out)
{
    c->stats = ejoin_stats{};
    if (!rel_ok(R) || !rel_ok(Q) || R.d != Q.d || !sel_ok(selR) || std::isnan(eps)) return EJOIN_EINVAL;
    const bool timing = (c->flags & EJOIN_FLAG_TIMING) != 0;
    const bool count_only = (c->flags & EJOIN_FLAG_COUNT_ONLY) != 0;
    const int64_t kp = ejoin_padded_dim(EJOIN_TF32, R.d);
    const float band = c->band_cfg >= 0.f ? c->band_cfg : default_band(EJOIN_TF32, kp);
    c->stats.band = band;
    const int64_t m = Q.n;
    const int64_t n_chunks = (m + 63) / 64;
    cudaError_t e;
    Side &sa = c->side[0];
    Side &sq = c->side[1];
    const int64_t qrows = std::max<int64_t>(n_chunks, 1) * 64;
    const int64_t rows = round_up(std::max<int64_t>(R.n, 1), 128);
    if ((e = ensure(sq.norm, (size_t)qrows * kp * 4)) != cudaSuccess) return from_cuda(e);
    if ((e = ensure(sq.inv, (size_t)qrows * 4)) != cudaSuccess) return from_cuda(e);
    if ((e = ensure(sa.inv, (size_t)rows * 4)) != cudaSuccess) return from_cuda(e);
    if (c->cand_cap == 0) c->cand_cap = c->cap_hint;
    if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
    DevMisc *dm = (DevMisc *)c->misc.p;
    bool direct = !selR && R.n > 0 && R.ld % 4 == 0 && (reinterpret_cast<uintptr_t>(R.x) & 15) == 0;

    for (int attempt = 0; attempt < 2; ++attempt) {
        c->stats.launches = 0;
        if ((e = cudaMemsetAsync(dm, 0, sizeof(DevMisc), c->stream)) != cudaSuccess) return from_cuda(e);
        if (timing) cudaEventRecord(c->ev[0], c->stream);
        ejoin_status st = prepare_side(c, 1, Q, nullptr, FMT_F32, kp, sq.norm.p, kp, (float *)sq.inv.p, nullptr,
                                       nullptr, &dm->n_sel[1], &dm->status, false);
        if (st != EJOIN_OK) return st;
        CUtensorMap tmR;
        if (direct) {
            if ((e = launch_set_count(&dm->n_sel[0], (long long)R.n, c->stream)) != cudaSuccess) return from_cuda(e);
            c->stats.launches += 1;
            if (!make_tmap_rows_f32(&tmR, R.x, R.d, R.ld, R.n, 128)) return EJOIN_ECUDA;
        } else {
            if ((e = ensure(sa.norm, (size_t)rows * kp * 4)) != cudaSuccess) return from_cuda(e);
            if (selR && (e = ensure(sa.ids, (size_t)rows * 4)) != cudaSuccess) return from_cuda(e);
            st = prepare_side(c, 0, R, selR, FMT_F32, kp, sa.norm.p, kp, (float *)sa.inv.p, nullptr,
                              (uint32_t *)sa.ids.p, &dm->n_sel[0], &dm->status, false);
            if (st != EJOIN_OK) return st;
            if (!make_tmap(&tmR, sa.norm.p, FMT_F32, kp, rows, 128)) return EJOIN_ECUDA;
        }
        if (timing) cudaEventRecord(c->ev[1], c->stream);
        auto scan = [&]() -> cudaError_t {
            for (int64_t ch = 0; ch < n_chunks; ++ch) {
                CUtensorMap tmQ;
                if (!make_tmap(&tmQ, (const char *)sq.norm.p + (size_t)ch * 64 * kp * 4, FMT_F32, kp, 64, 64))
                    return cudaErrorInvalidValue;
                const int mc = (int)std::min<int64_t>(64, m - ch * 64);
                cudaError_t ee = launch_esel(&tmR, &tmQ, (int)(kp / 32), &dm->n_sel[0], mc, (int)(ch * 64),
                                             eps - band, (direct && ch == 0) ? (float *)sa.inv.p : nullptr,
                                             (uint2 *)c->cand.p, c->cand_cap, &dm->cand_count, &dm->status,
                                             c->timeout, c->num_sms, c->stream);
                if (ee != cudaSuccess) return ee;
                c->stats.launches += 1;
            }
            return cudaSuccess;
        };
        if (m > 0 && R.n > 0 && (e = scan()) != cudaSuccess) return from_cuda(e);
        if (timing) cudaEventRecord(c->ev[2], c->stream);
        DevMisc hm;
        auto read_misc = [&]() -> cudaError_t {
            cudaError_t ee = cudaMemcpyAsync(&hm, dm, sizeof(DevMisc), cudaMemcpyDeviceToHost, c->stream);
            return ee == cudaSuccess ? cudaStreamSynchronize(c->stream) : ee;
        };
        if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
        if ((hm.status & ERR_RANGE) && !(hm.status & (ERR_NONFINITE | ERR_TIMEOUT)) && direct) {
            direct = false;  // a row needs the rescaling normalisation pass
            continue;
        }
        if (hm.status) return status_of(hm.status);
        c->stats.n_sel_r = (uint64_t)hm.n_sel[0];
        c->stats.n_sel_s = (uint64_t)m;
        while (hm.cand_count > c->cand_cap) {
            c->cand_cap = hm.cand_count + hm.cand_count / 4 + 1024;
            if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
            if ((e = cudaMemsetAsync(&dm->cand_count, 0, sizeof(unsigned long long), c->stream)) != cudaSuccess)
                return from_cuda(e);
            if ((e = scan()) != cudaSuccess) return from_cuda(e);
            if (timing) cudaEventRecord(c->ev[2], c->stream);
            if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
            if (hm.status) return status_of(hm.status);
            c->stats.contract_retries++;
        }
        c->stats.candidates = hm.cand_count;
        if (*pairs_io == nullptr && may_alloc && !count_only) {
            const uint64_t cap = std::max<uint64_t>(hm.cand_count, 1);
            void *p = nullptr;
            if ((e = cudaMalloc(&p, cap * sizeof(ejoin_pair))) != cudaSuccess) return from_cuda(e);
            *pairs_io = (ejoin_pair *)p;
            *cap_io = cap;
        }
        if (*pairs_io == nullptr && !count_only) *cap_io = 0;
        if ((e = ensure(c->band, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
        if (hm.cand_count) {
            e = launch_rescore((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, R.x, R.ld, Q.x, Q.ld, R.d,
                               (!direct && selR) ? (const uint32_t *)sa.ids.p : nullptr, nullptr,
                               (const float *)sa.inv.p, (const float *)sq.inv.p, eps, c->fp64_band, *pairs_io,
                               count_only ? 0 : *cap_io, &dm->pair_count, &dm->band_count, count_only ? 1 : 0,
                               c->num_sms, c->stream, (uint2 *)c->band.p, c->cand_cap, 0);
            if (e != cudaSuccess) return from_cuda(e);
            c->stats.launches += c->fp64_band > 0.f ? 2 : 1;
        }
        if (timing) cudaEventRecord(c->ev[3], c->stream);
        if ((e = read_misc()) != cudaSuccess) return from_cuda(e);
        if (hm.status) return status_of(hm.status);
        c->stats.pairs = hm.pair_count;
        c->stats.fp64_rescored = hm.band_count;
        if (timing) {
            c->stats.ms_normalize = elapsed(c->ev[0], c->ev[1]);
            c->stats.ms_contract = elapsed(c->ev[1], c->ev[2]);
            c->stats.ms_rescore = elapsed(c->ev[2], c->ev[3]);
            c->stats.ms_total = elapsed(c->ev[0], c->ev[3]);
        }
        c->stats.fused = direct ? 1 : 0;
        *count_out = hm.pair_count;
        if (!count_only && hm.pair_count > *cap_io) return EJOIN_EOVERFLOW;
        if ((c->flags & EJOIN_FLAG_SORT) && !count_only) return sort_result(c, *pairs_io, hm.pair_count, R.n, Q.n);
        return EJOIN_OK;
    }
    return EJOIN_ECUDA;
}

}  // namespace

extern "C" {

ejoin_status ejoin_threshold(ejoin_ctx *c, ejoin_rel R, ejoin_rel S, float eps, const ejoin_sel *selR,
                             const ejoin_sel *selS, ejoin_pairs *out)
{
    if (!c || !out) return EJOIN_EINVAL;
    DeviceGuard g(c->device);
    uint64_t count = 0;
    ejoin_pair *p = out->d_pairs;
    uint64_t cap = out->capacity;
    const bool alloc = p == nullptr;
    ejoin_status st = run_threshold(c, R, S, eps, selR, selS, &p, &cap, alloc, out->d_count, &count);
    if (alloc && p) {
        out->d_pairs = p;
        out->capacity = cap;
    }
    out->count = count;
    return st;
}

ejoin_status ejoin_topk(ejoin_ctx *c, ejoin_rel R, ejoin_rel S, int32_t k, const ejoin_sel *selR,
                        const ejoin_sel *selS, ejoin_pairs *out)
{
    if (!c || !out) return EJOIN_EINVAL;
    DeviceGuard g(c->device);
    uint64_t count = 0;
    ejoin_pair *p = out->d_pairs;
    uint64_t cap = out->capacity;
    const bool alloc = p == nullptr;
    ejoin_status st = run_topk(c, R, S, k, selR, selS, &p, &cap, alloc, &count);
    if (alloc && p) {
        out->d_pairs = p;
        out->capacity = cap;
    }
    out->count = count;
    if (out->d_count && (st == EJOIN_OK || st == EJOIN_EOVERFLOW)) {
        const uint64_t cnt = count;
        if (cudaMemcpyAsync(out->d_count, &cnt, sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return EJOIN_ECUDA;
    }
    return st;
}

ejoin_status ejoin_eselect(ejoin_ctx *c, ejoin_rel R, const ejoin_sel *selR, ejoin_rel Q, float eps,
                           ejoin_pairs *out)
{
    if (!c || !out) return EJOIN_EINVAL;
    DeviceGuard g(c->device);
    uint64_t count = 0;
    ejoin_pair *p = out->d_pairs;
    uint64_t cap = out->capacity;
    const bool alloc = p == nullptr;
    ejoin_status st = run_eselect(c, R, selR, Q, eps, &p, &cap, alloc, &count);
    if (alloc && p) {
        out->d_pairs = p;
        out->capacity = cap;
    }
    out->count = count;
    if (out->d_count && (st == EJOIN_OK || st == EJOIN_EOVERFLOW)) {
        const uint64_t cnt = count;
        if (cudaMemcpyAsync(out->d_count, &cnt, sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return EJOIN_ECUDA;
    }
    return st;
}

ejoin_status ejoin_top1(ejoin_ctx *c, ejoin_rel R, ejoin_rel S, const ejoin_sel *selR, const ejoin_sel *selS,
                        ejoin_pairs *out)
{
    return ejoin_topk(c, R, S, 1, selR, selS, out);
}

ejoin_status ejoin_threshold_host(ejoin_ctx *c, ejoin_rel R, ejoin_rel S, float eps, const ejoin_sel *selR,
                                  const ejoin_sel *selS, ejoin_pair *h_pairs, uint64_t capacity, uint64_t *count)
{
    if (!c || !count || (capacity && !h_pairs)) return EJOIN_EINVAL;
    if (!rel_ok(R) || !rel_ok(S) || R.d != S.d || !sel_ok(selR) || !sel_ok(selS)) return EJOIN_EINVAL;
    DeviceGuard g(c->device);
    const bool timing = (c->flags & EJOIN_FLAG_TIMING) != 0;
    cudaError_t e;
    const bool self = R.x == S.x && R.n == S.n && R.ld == S.ld && same_sel(selR, selS);
    // the device address of a host buffer the kernels can read in place (pinned memory), else nullptr
    auto in_place = [](const void *h) -> const void * {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
            cudaGetLastError();  // not a CUDA-known pointer: clear the error
            return nullptr;
        }
        return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
    };
    bool zc = (c->flags & EJOIN_FLAG_HOST_COPY) == 0;
    const void *zR = nullptr, *zS = nullptr, *zRa = nullptr, *zRb = nullptr, *zSa = nullptr, *zSb = nullptr;
    if (zc && R.n > 0) zc = (zR = in_place(R.x)) != nullptr;
    if (zc && S.n > 0) zc = (zS = in_place(S.x)) != nullptr;
    if (zc && selR && selR->attr && R.n > 0) zc = (zRa = in_place(selR->attr)) != nullptr;
    if (zc && selR && selR->bits && R.n > 0) zc = (zRb = in_place(selR->bits)) != nullptr;
    if (zc && selS && selS->attr && S.n > 0) zc = (zSa = in_place(selS->attr)) != nullptr;
    if (zc && selS && selS->bits && S.n > 0) zc = (zSb = in_place(selS->bits)) != nullptr;
    if (timing) cudaEventRecord(c->ev[4], c->stream);
    ejoin_rel dR, dS;
    ejoin_sel dsR, dsS;
    float *rawR = nullptr, *rawS = nullptr;
    uint64_t h2d = 0;
    if (zc) {
        // kernels read the host buffers in place; the kept rows are copied to the device by the
        // normalisation pass (the re-score gathers them there)
        dR = R;
        dR.x = (const float *)zR;
        dS = S;
        dS.x = self ? dR.x : (const float *)zS;
        if (R.n > 0) {
            if ((e = ensure(c->host_in[0], (size_t)R.n * R.d * 4)) != cudaSuccess) return from_cuda(e);
            rawR = (float *)c->host_in[0].p;
        }
        if (self) {
            rawS = rawR;
        } else if (S.n > 0) {
            if ((e = ensure(c->host_in[1], (size_t)S.n * S.d * 4)) != cudaSuccess) return from_cuda(e);
            rawS = (float *)c->host_in[1].p;
        }
        if (selR) {
            dsR = *selR;
            if (zRa) dsR.attr = (const int32_t *)zRa;
            if (zRb) dsR.bits = (const uint32_t *)zRb;
        }
        if (selS) {
            dsS = *selS;
            if (zSa) dsS.attr = (const int32_t *)zSa;
            if (zSb) dsS.bits = (const uint32_t *)zSb;
        }
    } else {
        // host -> device copies of the inputs (rows are copied densely: ld = d)
        auto up_rel = [&](int slot, const ejoin_rel &r, ejoin_rel &dr) -> cudaError_t {
            dr = r;
            dr.ld = r.d;
            if (r.n == 0) {
                dr.x = nullptr;
                return cudaSuccess;
            }
            cudaError_t ee = ensure(c->host_in[slot], (size_t)r.n * r.d * 4);
            if (ee != cudaSuccess) return ee;
            dr.x = (const float *)c->host_in[slot].p;
            h2d += (uint64_t)r.n * r.d * 4;
            if (r.ld == r.d)
                return cudaMemcpyAsync(c->host_in[slot].p, r.x, (size_t)r.n * r.d * 4, cudaMemcpyHostToDevice,
                                       c->stream);
            return cudaMemcpy2DAsync(c->host_in[slot].p, (size_t)r.d * 4, r.x, (size_t)r.ld * 4, (size_t)r.d * 4,
                                     (size_t)r.n, cudaMemcpyHostToDevice, c->stream);
        };
        auto up_sel = [&](int slot, const ejoin_sel *s, int64_t n, ejoin_sel &ds) -> cudaError_t {
            ds = *s;
            const size_t abytes = s->attr ? (size_t)n * 4 : 0;
            const size_t bbytes = s->bits ? (size_t)((n + 31) / 32) * 4 : 0;
            cudaError_t ee = ensure(c->host_in[slot], abytes + bbytes + 16);
            if (ee != cudaSuccess) return ee;
            char *base = (char *)c->host_in[slot].p;
            if (s->attr && n) {
                if ((ee = cudaMemcpyAsync(base, s->attr, abytes, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
                    return ee;
                ds.attr = (const int32_t *)base;
                h2d += abytes;
            }
            if (s->bits && n) {
                char *bb = base + ((abytes + 15) & ~size_t(15));
                if ((ee = cudaMemcpyAsync(bb, s->bits, bbytes, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
                    return ee;
                ds.bits = (const uint32_t *)bb;
                h2d += bbytes;
            }
            return cudaSuccess;
        };
        if ((e = up_rel(0, R, dR)) != cudaSuccess) return from_cuda(e);
        if (self) {
            dS = dR;
        } else if ((e = up_rel(1, S, dS)) != cudaSuccess) {
            return from_cuda(e);
        }
        if (selR && (e = up_sel(2, selR, R.n, dsR)) != cudaSuccess) return from_cuda(e);
        if (selS) {
            if (self) {
                dsS = dsR;
            } else if ((e = up_sel(3, selS, S.n, dsS)) != cudaSuccess) {
                return from_cuda(e);
            }
        }
    }
    if (timing) cudaEventRecord(c->ev[5], c->stream);
    // a pinned result buffer is written by the re-score in place; otherwise through a device buffer
    ejoin_pair *dp = nullptr;
    if (zc && capacity) dp = (ejoin_pair *)in_place(h_pairs);
    const bool out_in_place = dp != nullptr;
    if (!out_in_place) {
        if ((e = ensure(c->host_pairs, std::max<uint64_t>(capacity, 1) * sizeof(ejoin_pair))) != cudaSuccess)
            return from_cuda(e);
        dp = (ejoin_pair *)c->host_pairs.p;
    }
    uint64_t cap = capacity;
    uint64_t cnt = 0;
    ejoin_status st = run_threshold(c, dR, dS, eps, selR ? &dsR : nullptr, selS ? &dsS : nullptr, &dp, &cap, false,
                                    nullptr, &cnt, rawR, rawS);
    *count = cnt;
    if (zc) {
        // what the kernels read from host memory: the kept rows and the predicate columns
        h2d = c->stats.n_sel_r * (uint64_t)R.d * 4 + (self ? 0 : c->stats.n_sel_s * (uint64_t)S.d * 4);
        if (selR) h2d += (selR->attr ? (uint64_t)R.n * 4 : 0) + (selR->bits ? (uint64_t)((R.n + 31) / 32) * 4 : 0);
        if (selS && !self)
            h2d += (selS->attr ? (uint64_t)S.n * 4 : 0) + (selS->bits ? (uint64_t)((S.n + 31) / 32) * 4 : 0);
    }
    c->stats.h2d_bytes = h2d;
    c->stats.host_in_place = zc ? 1 : 0;
    if (st != EJOIN_OK && st != EJOIN_EOVERFLOW) return st;
    const uint64_t ncopy = std::min<uint64_t>(cnt, capacity);
    if (timing) cudaEventRecord(c->ev[6], c->stream);
    if (ncopy && !out_in_place && (c->flags & EJOIN_FLAG_COUNT_ONLY) == 0) {
        if ((e = cudaMemcpyAsync(h_pairs, dp, ncopy * sizeof(ejoin_pair), cudaMemcpyDeviceToHost, c->stream)) !=
            cudaSuccess)
            return from_cuda(e);
    }
    if (timing) cudaEventRecord(c->ev[7], c->stream);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return from_cuda(e);
    if (timing) {
        c->stats.ms_h2d = elapsed(c->ev[4], c->ev[5]);
        c->stats.ms_d2h = elapsed(c->ev[6], c->ev[7]);
    }
    return st;
}

ejoin_status ejoin_normalize(ejoin_ctx *c, ejoin_rel in, const ejoin_sel *sel, int32_t prec, void *d_out,
                             int64_t ld_out, float *d_inv_norm, float *d_scale, uint32_t *d_ids, int64_t *d_n_sel)
{
    if (!c || !rel_ok(in) || !sel_ok(sel) || !d_out || !d_n_sel) return EJOIN_EINVAL;
    if (prec < EJOIN_F32 || prec > EJOIN_TF32) return EJOIN_EINVAL;
    const int64_t kp = ejoin_padded_dim(prec, in.d);
    if (ld_out < kp) return EJOIN_EINVAL;
    const int fmt = fmt_of(prec);
    if (fmt == FMT_FP8 && !d_scale) return EJOIN_EINVAL;
    // vector stores of 4 elements per lane: 16-byte (F32), 8-byte (BF16), 4-byte (e4m3) alignment
    if ((ld_out & 3) || (reinterpret_cast<uintptr_t>(d_out) & (4 * fmt_bytes(fmt) - 1))) return EJOIN_EINVAL;
    DeviceGuard g(c->device);
    cudaError_t e;
    Side &sd = c->side[0];
    uint32_t *ids = d_ids;
    if (sel && !ids) {
        if ((e = ensure(sd.ids, (size_t)std::max<int64_t>(in.n, 1) * 4)) != cudaSuccess) return from_cuda(e);
        ids = (uint32_t *)sd.ids.p;
    }
    DevMisc *dm = (DevMisc *)c->misc.p;
    return prepare_side(c, 0, in, sel, fmt, kp, d_out, ld_out, d_inv_norm, d_scale, ids, (long long *)d_n_sel,
                        &dm->status, false);
}

}  // extern "C"
