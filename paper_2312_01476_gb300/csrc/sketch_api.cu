// C ABI of the learned part: the sketch network (parameters, forward,
// gradient, Adam step, pair scoring) and the pruned join that uses its
// sketches to skip tile pairs.  The paper has no learned component; these
// entry points implement the "learned tile pruning" form of the join.
//
// Pruned join (ejoin_threshold_pruned), all on the context stream:
//   1. normalise R and S (BF16 operands, FP32 inverse norms), as in the plain join;
//   2. sketch every row with the network (unit 64-d vectors);
//   3. reorder each side so that tiles are coherent in sketch space: covering
//      anchors drawn in rounds from a sample (prune.cu), every row joins its
//      most similar anchor, counting sort by anchor, gather of operand rows,
//      inverse norms and sketches;
//   4. per tile: up to 4 balls in sketch space (seeds by farthest-point
//      sampling in the tile, rows join the nearest seed: unit centroid +
//      angular radius); a tile pair is kept when some
//      ball pair has cos(max(0, angle - rho_a - rho_b)) >= eps_sketch; kept
//      pairs are compacted into a tile list;
//   5. the tcgen05 contraction runs on the listed tiles only (threshold eps -
//      band), and the re-score verifies every candidate exactly from the FP32
//      input rows, mapping sorted rows back to original ids.
#include <cstring>
#include <new>
#include <vector>

#include "host_internal.h"
#include "mlp_internal.cuh"

using namespace ej;
using namespace ej::host;

struct ejoin_sketch {
    ejoin_ctx *ctx = nullptr;
    int device = 0;  // the context's device, kept for teardown
    int d = 0, hid = 0, out = 0;
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, n_params = 0;
    Buf params, grads, m, v;
    int step = 0;
    // training workspace (grown on demand)
    Buf idx, A1, H, Z, S, nz, dS, dZ, dH, scal;  // scal: [loss, wsum]
    // forward workspace
    Buf fH, fZ, finv, fcnt;
    // pruned-join workspace, per side
    struct Side {
        Buf S, key1, perm1, perm, hist, a_idx, anchors2, norm, inv, scale, sS, maxdot, cent, rad;
        Buf skb, anb, tinv, best, cnt;  // assignment contraction: BF16 sketches and anchors, argmax
        Buf smpb, rab;                  // covering rounds: BF16 sketches of the sample and of a round's anchors
        int n_anchor = 0;               // covering anchors of the last reorder
    } pw[2];
    Buf list, list_count;
    uint64_t list_cap = 0;
    // tile-pair bounds on the tensor cores: augmented ball rows of both sides, kept ball pairs, bitmap
    Buf ballA, ballB, bcand, bmisc, bits, rowcnt;
    uint64_t bcand_cap = 0;
};

namespace {

constexpr int64_t FWD_CHUNK = 1 << 20;

cudaError_t grow(Buf &b, size_t bytes) { return ensure(b, bytes); }

float *P(Buf &b) { return (float *)b.p; }

// The same forward with both layers on the tensor cores (TF32 from the FP32 operands, FP32 accumulation):
// H = GELU(inv * X W1^T + b1), Z = H W2^T + b2, rows of Z normalised.  The products carry TF32 rounding
// (relative 2^-10 per operand element) instead of FP32's, a sketch-cosine error of about 1e-3, well inside
// the calibration margin; the pruned join uses it for its sketches.  cudaErrorNotSupported when the
// layout does not allow tensor maps (the caller then uses sketch_forward).
cudaError_t sketch_forward_tc(ejoin_sketch *sk, const float *x, int64_t n, int64_t ld, const float *inv, float *S_out,
                              cudaStream_t st)
{
    ejoin_ctx *c = sk->ctx;
    const float *W = P(sk->params);
    const int d = sk->d, hid = sk->hid, out = sk->out;
    if (ld % 4 || d % 4 || hid % 4 || (reinterpret_cast<uintptr_t>(x) & 15) || (sk->oW2 % 4) || (sk->ob1 % 4))
        return cudaErrorNotSupported;
    cudaError_t e;
    const int64_t chunk = std::min<int64_t>(n, FWD_CHUNK);
    if ((e = grow(sk->fH, (size_t)std::max<int64_t>(chunk, 1) * hid * 4)) ||
        (e = grow(sk->fZ, (size_t)std::max<int64_t>(chunk, 1) * out * 4)) || (e = grow(sk->fcnt, 64)))
        return e;
    long long *cnt = (long long *)sk->fcnt.p;  // [0] rows of the chunk, [1] hid, [2] out
    if ((e = launch_set_count(cnt + 1, hid, st)) || (e = launch_set_count(cnt + 2, out, st))) return e;
    CUtensorMap tW1, tW2, tH;
    if (!make_tmap_rows_f32(&tW1, W + sk->oW1, d, d, hid, 256) ||
        !make_tmap_rows_f32(&tW2, W + sk->oW2, hid, hid, out, 256) ||
        !make_tmap_rows_f32(&tH, P(sk->fH), hid, hid, std::max<int64_t>(chunk, 1), 128))
        return cudaErrorNotSupported;
    DevMisc *dm = (DevMisc *)c->misc.p;
    const int kp1 = (int)round_up(d, 32), kp2 = (int)round_up(hid, 32);
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t m = std::min<int64_t>(chunk, n - r0);
        CUtensorMap tX;
        if (!make_tmap_rows_f32(&tX, x + r0 * ld, d, ld, m, 128)) return cudaErrorNotSupported;
        if ((e = launch_set_count(cnt, m, st)) ||
            (e = launch_gemm_tc(&tX, &tW1, kp1, cnt, cnt + 1, inv + r0, W + sk->ob1, ACT_GELU, P(sk->fH), hid,
                                &dm->status, c->timeout, c->num_sms, st)) ||
            (e = launch_gemm_tc(&tH, &tW2, kp2, cnt, cnt + 2, nullptr, W + sk->ob2, ACT_NONE, P(sk->fZ), out,
                                &dm->status, c->timeout, c->num_sms, st)) ||
            (e = launch_rownorm(P(sk->fZ), m, out, S_out + r0 * out, nullptr, c->num_sms, st)))
            return e;
    }
    return cudaSuccess;
}

// Forward of rows [0, n) of x (raw rows; inv = their inverse norms) into S_out (n x out).
cudaError_t sketch_forward(ejoin_sketch *sk, const float *x, int64_t n, int64_t ld, const float *inv, float *S_out,
                           cudaStream_t st)
{
    ejoin_ctx *c = sk->ctx;
    cudaError_t e;
    const int64_t chunk = std::min<int64_t>(n, FWD_CHUNK);
    if ((e = grow(sk->fH, (size_t)std::max<int64_t>(chunk, 1) * sk->hid * 4)) != cudaSuccess) return e;
    if ((e = grow(sk->fZ, (size_t)std::max<int64_t>(chunk, 1) * sk->out * 4)) != cudaSuccess) return e;
    float *W = P(sk->params);
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t m = std::min<int64_t>(chunk, n - r0);
        // the inference-form GEMM where the layout allows it, else the generic one
        e = launch_gemm_nt_f32(x + r0 * ld, ld, W + sk->oW1, sk->d, W + sk->ob1, inv + r0, ACT_GELU, P(sk->fH),
                               sk->hid, m, sk->hid, sk->d, st);
        if (e == cudaErrorInvalidValue) {
            cudaGetLastError();
            GemmArgs g1;
            g1.A = x + r0 * ld;
            g1.a_rs = ld;
            g1.a_cs = 1;
            g1.B = W + sk->oW1;
            g1.b_rs = 1;
            g1.b_cs = sk->d;
            g1.C = P(sk->fH);
            g1.ldc = sk->hid;
            g1.bias = W + sk->ob1;
            g1.rowscale = inv + r0;
            g1.M = m;
            g1.N = sk->hid;
            g1.K = sk->d;
            g1.act = ACT_GELU;
            e = launch_gemm_f32(g1, c->num_sms, st);
        }
        if (e != cudaSuccess) return e;
        e = launch_gemm_nt_f32(P(sk->fH), sk->hid, W + sk->oW2, sk->hid, W + sk->ob2, nullptr, ACT_NONE, P(sk->fZ),
                               sk->out, m, sk->out, sk->hid, st);
        if (e == cudaErrorInvalidValue) {
            cudaGetLastError();
            GemmArgs g2;
            g2.A = P(sk->fH);
            g2.a_rs = sk->hid;
            g2.a_cs = 1;
            g2.B = W + sk->oW2;
            g2.b_rs = 1;
            g2.b_cs = sk->hid;
            g2.C = P(sk->fZ);
            g2.ldc = sk->out;
            g2.bias = W + sk->ob2;
            g2.M = m;
            g2.N = sk->out;
            g2.K = sk->hid;
            e = launch_gemm_f32(g2, c->num_sms, st);
        }
        if (e != cudaSuccess) return e;
        if ((e = launch_rownorm(P(sk->fZ), m, sk->out, S_out + r0 * sk->out, nullptr, c->num_sms, st)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// Forward + backward on a batch of pairs (rows p[k], q[k] of x); gradients into sk->grads.
cudaError_t sketch_grad(ejoin_sketch *sk, const float *x, int64_t ld, const float *inv, const uint32_t *p,
                        const uint32_t *q, const float *t, const float *w, int64_t B, cudaStream_t st)
{
    ejoin_ctx *c = sk->ctx;
    const int64_t n = 2 * B;
    const int hid = sk->hid, out = sk->out, d = sk->d;
    cudaError_t e;
    if ((e = grow(sk->idx, (size_t)n * 4)) || (e = grow(sk->A1, (size_t)n * hid * 4)) ||
        (e = grow(sk->H, (size_t)n * hid * 4)) || (e = grow(sk->Z, (size_t)n * out * 4)) ||
        (e = grow(sk->S, (size_t)n * out * 4)) || (e = grow(sk->nz, (size_t)n * 4)) ||
        (e = grow(sk->dS, (size_t)n * out * 4)) || (e = grow(sk->dZ, (size_t)n * out * 4)) ||
        (e = grow(sk->dH, (size_t)n * hid * 4)) || (e = grow(sk->scal, 64)))
        return e;
    uint32_t *idx = (uint32_t *)sk->idx.p;
    if ((e = cudaMemcpyAsync(idx, p, B * 4, cudaMemcpyDeviceToDevice, st)) ||
        (e = cudaMemcpyAsync(idx + B, q, B * 4, cudaMemcpyDeviceToDevice, st)))
        return e;
    float *W = P(sk->params), *G = P(sk->grads);
    // forward
    GemmArgs g1;
    g1.A = x;
    g1.aidx = idx;
    g1.a_rs = ld;
    g1.a_cs = 1;
    g1.B = W + sk->oW1;
    g1.b_rs = 1;
    g1.b_cs = d;
    g1.C = P(sk->H);
    g1.ldc = hid;
    g1.bias = W + sk->ob1;
    g1.rowscale = inv;
    g1.pre = P(sk->A1);
    g1.M = n;
    g1.N = hid;
    g1.K = d;
    g1.act = ACT_GELU;
    if ((e = launch_gemm_f32(g1, c->num_sms, st)) != cudaSuccess) return e;
    GemmArgs g2;
    g2.A = P(sk->H);
    g2.a_rs = hid;
    g2.a_cs = 1;
    g2.B = W + sk->oW2;
    g2.b_rs = 1;
    g2.b_cs = hid;
    g2.C = P(sk->Z);
    g2.ldc = out;
    g2.bias = W + sk->ob2;
    g2.M = n;
    g2.N = out;
    g2.K = hid;
    if ((e = launch_gemm_f32(g2, c->num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_rownorm(P(sk->Z), n, out, P(sk->S), P(sk->nz), c->num_sms, st)) != cudaSuccess) return e;
    // loss and dL/ds
    float *scal = P(sk->scal);
    if ((e = cudaMemsetAsync(scal, 0, 64, st)) != cudaSuccess) return e;
    if ((e = launch_colsum(w, B, 1, scal + 1, c->num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_pair_grad(P(sk->S), B, out, t, w, scal + 1, P(sk->dS), scal, c->num_sms, st)) != cudaSuccess)
        return e;
    // backward
    if ((e = launch_rownorm_backward(P(sk->S), P(sk->dS), P(sk->nz), n, out, P(sk->dZ), c->num_sms, st)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(G, 0, (size_t)sk->n_params * 4, st)) != cudaSuccess) return e;
    GemmArgs gw2;  // dW2 = dZ^T H
    gw2.A = P(sk->dZ);
    gw2.a_rs = 1;
    gw2.a_cs = out;
    gw2.B = P(sk->H);
    gw2.b_rs = hid;
    gw2.b_cs = 1;
    gw2.C = G + sk->oW2;
    gw2.ldc = hid;
    gw2.M = out;
    gw2.N = hid;
    gw2.K = n;
    gw2.atomic_acc = 1;
    if ((e = launch_gemm_f32(gw2, c->num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_colsum(P(sk->dZ), n, out, G + sk->ob2, c->num_sms, st)) != cudaSuccess) return e;
    GemmArgs gh;  // dH = dZ W2
    gh.A = P(sk->dZ);
    gh.a_rs = out;
    gh.a_cs = 1;
    gh.B = W + sk->oW2;
    gh.b_rs = hid;
    gh.b_cs = 1;
    gh.C = P(sk->dH);
    gh.ldc = hid;
    gh.M = n;
    gh.N = hid;
    gh.K = out;
    if ((e = launch_gemm_f32(gh, c->num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_gelu_backward(P(sk->dH), P(sk->A1), n * hid, c->num_sms, st)) != cudaSuccess) return e;
    GemmArgs gw1;  // dW1 = dA1^T X (rows gathered and scaled to unit length)
    gw1.A = P(sk->dH);
    gw1.a_rs = 1;
    gw1.a_cs = hid;
    gw1.B = x;
    gw1.bidx = idx;
    gw1.bscale = inv;
    gw1.b_rs = ld;
    gw1.b_cs = 1;
    gw1.C = G + sk->oW1;
    gw1.ldc = d;
    gw1.M = hid;
    gw1.N = d;
    gw1.K = n;
    gw1.atomic_acc = 1;
    if ((e = launch_gemm_f32(gw1, c->num_sms, st)) != cudaSuccess) return e;
    return launch_colsum(P(sk->dH), n, hid, G + sk->ob1, c->num_sms, st);
}

ejoin_status check_pairs_args(const ejoin_sketch *sk, ejoin_rel X, const float *inv, const uint32_t *p,
                              const uint32_t *q, const float *t, const float *w, int64_t B)
{
    if (!sk || !X.x || X.d != sk->d || X.ld < X.d || X.n <= 0 || !inv || !p || !q || B <= 0) return EJOIN_EINVAL;
    if ((t == nullptr) != (w == nullptr)) return EJOIN_EINVAL;
    return EJOIN_OK;
}

}  // namespace

extern "C" {

ejoin_status ejoin_sketch_create(ejoin_ctx *ctx, int32_t d, int32_t hidden, int32_t out, ejoin_sketch **res)
{
    if (!ctx || !res || d < 1 || d > 4096 || hidden < 1 || hidden > 4096 || out != 64) return EJOIN_EINVAL;
    *res = nullptr;
    DeviceGuard g(ctx->device);
    ejoin_sketch *sk = new (std::nothrow) ejoin_sketch();
    if (!sk) return EJOIN_ENOMEM;
    sk->ctx = ctx;
    sk->device = ctx->device;
    sk->d = d;
    sk->hid = hidden;
    sk->out = out;
    sk->oW1 = 0;
    sk->ob1 = (int64_t)hidden * d;
    sk->oW2 = sk->ob1 + hidden;
    sk->ob2 = sk->oW2 + (int64_t)out * hidden;
    sk->n_params = sk->ob2 + out;
    cudaError_t e;
    const size_t bytes = (size_t)sk->n_params * 4;
    if ((e = ensure(sk->params, bytes)) || (e = ensure(sk->grads, bytes)) || (e = ensure(sk->m, bytes)) ||
        (e = ensure(sk->v, bytes))) {
        ejoin_sketch_destroy(sk);
        return from_cuda(e);
    }
    *res = sk;
    return EJOIN_OK;
}

void ejoin_sketch_destroy(ejoin_sketch *sk)
{
    if (!sk) return;
    {
        // the context may already be gone: wait for the device, not for its stream
        DeviceGuard g(sk->device);
        cudaDeviceSynchronize();
        for (Buf *b : {&sk->params, &sk->grads, &sk->m, &sk->v, &sk->idx, &sk->A1, &sk->H, &sk->Z, &sk->S, &sk->nz,
                       &sk->dS, &sk->dZ, &sk->dH, &sk->scal, &sk->fH, &sk->fZ, &sk->finv, &sk->fcnt, &sk->list,
                       &sk->list_count, &sk->ballA, &sk->ballB, &sk->bcand, &sk->bmisc, &sk->bits, &sk->rowcnt})
            release(*b);
        for (auto &w : sk->pw)
            for (Buf *b : {&w.S, &w.key1, &w.perm1, &w.perm, &w.hist, &w.a_idx, &w.anchors2, &w.norm, &w.inv,
                           &w.scale, &w.sS, &w.maxdot, &w.cent, &w.rad, &w.skb, &w.anb, &w.tinv, &w.best, &w.cnt,
                           &w.smpb, &w.rab})
                release(*b);
    }
    delete sk;
}

int64_t ejoin_sketch_num_params(const ejoin_sketch *sk) { return sk ? sk->n_params : 0; }

ejoin_status ejoin_sketch_set_params(ejoin_sketch *sk, const float *h_params)
{
    if (!sk || !h_params) return EJOIN_EINVAL;
    DeviceGuard g(sk->ctx->device);
    const size_t bytes = (size_t)sk->n_params * 4;
    cudaError_t e = cudaMemcpy(sk->params.p, h_params, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(sk->m.p, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(sk->v.p, 0, bytes);
    sk->step = 0;
    return from_cuda(e);
}

ejoin_status ejoin_sketch_get_params(const ejoin_sketch *sk, float *h_params)
{
    if (!sk || !h_params) return EJOIN_EINVAL;
    DeviceGuard g(sk->ctx->device);
    cudaError_t e = cudaStreamSynchronize(sk->ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h_params, sk->params.p, (size_t)sk->n_params * 4, cudaMemcpyDeviceToHost);
    return from_cuda(e);
}

ejoin_status ejoin_sketch_forward(ejoin_sketch *sk, ejoin_rel X, float *d_S)
{
    if (!sk || !d_S || X.d != sk->d || X.ld < X.d || X.n < 0 || (X.n && !X.x)) return EJOIN_EINVAL;
    if (X.n == 0) return EJOIN_OK;
    DeviceGuard g(sk->ctx->device);
    cudaError_t e = ensure(sk->finv, (size_t)X.n * 4);
    if (e == cudaSuccess) e = launch_row_inv_norm(X.x, X.n, X.d, X.ld, P(sk->finv), sk->ctx->num_sms, sk->ctx->stream);
    if (e == cudaSuccess) e = sketch_forward(sk, X.x, X.n, X.ld, P(sk->finv), d_S, sk->ctx->stream);
    return from_cuda(e);
}

ejoin_status ejoin_sketch_forward_tc(ejoin_sketch *sk, ejoin_rel X, float *d_S)
{
    if (!sk || !d_S || X.d != sk->d || X.ld < X.d || X.n < 0 || (X.n && !X.x)) return EJOIN_EINVAL;
    if (X.n == 0) return EJOIN_OK;
    DeviceGuard g(sk->ctx->device);
    cudaError_t e = ensure(sk->finv, (size_t)X.n * 4);
    if (e == cudaSuccess) e = launch_row_inv_norm(X.x, X.n, X.d, X.ld, P(sk->finv), sk->ctx->num_sms, sk->ctx->stream);
    if (e == cudaSuccess) e = sketch_forward_tc(sk, X.x, X.n, X.ld, P(sk->finv), d_S, sk->ctx->stream);
    if (e == cudaErrorNotSupported) return EJOIN_EUNSUPPORTED;
    return from_cuda(e);
}

ejoin_status ejoin_row_inv_norm(ejoin_ctx *ctx, ejoin_rel X, float *d_inv)
{
    if (!ctx || !d_inv || X.n < 0 || (X.n && !X.x) || X.ld < X.d) return EJOIN_EINVAL;
    DeviceGuard g(ctx->device);
    return from_cuda(launch_row_inv_norm(X.x, X.n, X.d, X.ld, d_inv, ctx->num_sms, ctx->stream));
}

ejoin_status ejoin_score_pairs(ejoin_ctx *ctx, ejoin_rel R, ejoin_rel S, const uint32_t *d_i, const uint32_t *d_j,
                               int64_t n_pairs, float *d_sim)
{
    if (!ctx || R.d != S.d || R.ld < R.d || S.ld < S.d || n_pairs < 0 || (n_pairs && (!d_i || !d_j || !d_sim)) ||
        (R.n && !R.x) || (S.n && !S.x))
        return EJOIN_EINVAL;
    if (n_pairs == 0) return EJOIN_OK;
    DeviceGuard g(ctx->device);
    Side &a = ctx->side[0], &b = ctx->side[1];
    cudaError_t e;
    if ((e = ensure(a.inv, (size_t)std::max<int64_t>(R.n, 1) * 4)) ||
        (e = ensure(b.inv, (size_t)std::max<int64_t>(S.n, 1) * 4)) ||
        (e = launch_row_inv_norm(R.x, R.n, R.d, R.ld, (float *)a.inv.p, ctx->num_sms, ctx->stream)) ||
        (e = launch_row_inv_norm(S.x, S.n, S.d, S.ld, (float *)b.inv.p, ctx->num_sms, ctx->stream)) ||
        (e = launch_score_pairs(R.x, R.ld, S.x, S.ld, R.d, d_i, d_j, (const float *)a.inv.p, (const float *)b.inv.p,
                                n_pairs, d_sim, ctx->num_sms, ctx->stream)))
        return from_cuda(e);
    return EJOIN_OK;
}

ejoin_status ejoin_sketch_grad(ejoin_sketch *sk, ejoin_rel X, const float *d_inv, const uint32_t *d_p,
                               const uint32_t *d_q, const float *d_t, const float *d_w, int64_t n_pairs,
                               float *d_grad, float *h_loss)
{
    ejoin_status s = check_pairs_args(sk, X, d_inv, d_p, d_q, d_t, d_w, n_pairs);
    if (s != EJOIN_OK || !d_t) return s != EJOIN_OK ? s : EJOIN_EINVAL;
    DeviceGuard g(sk->ctx->device);
    cudaStream_t st = sk->ctx->stream;
    cudaError_t e = sketch_grad(sk, X.x, X.ld, d_inv, d_p, d_q, d_t, d_w, n_pairs, st);
    if (e == cudaSuccess && d_grad)
        e = cudaMemcpyAsync(d_grad, sk->grads.p, (size_t)sk->n_params * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && h_loss) {
        e = cudaMemcpyAsync(h_loss, sk->scal.p, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return from_cuda(e);
}

ejoin_status ejoin_sketch_train_step(ejoin_sketch *sk, ejoin_rel X, const float *d_inv, const uint32_t *d_p,
                                     const uint32_t *d_q, const float *d_t, const float *d_w, int64_t n_pairs,
                                     float lr, float *h_loss)
{
    ejoin_status s = check_pairs_args(sk, X, d_inv, d_p, d_q, d_t, d_w, n_pairs);
    if (s != EJOIN_OK || !d_t) return s != EJOIN_OK ? s : EJOIN_EINVAL;
    DeviceGuard g(sk->ctx->device);
    cudaStream_t st = sk->ctx->stream;
    cudaError_t e = sketch_grad(sk, X.x, X.ld, d_inv, d_p, d_q, d_t, d_w, n_pairs, st);
    if (e != cudaSuccess) return from_cuda(e);
    sk->step += 1;
    e = launch_adam(P(sk->params), P(sk->grads), P(sk->m), P(sk->v), sk->n_params, lr, 0.9f, 0.999f, 1e-8f,
                    sk->step, sk->ctx->num_sms, st);
    if (e == cudaSuccess && h_loss) {
        e = cudaMemcpyAsync(h_loss, sk->scal.p, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return from_cuda(e);
}

ejoin_status ejoin_sketch_pair_sims(ejoin_sketch *sk, ejoin_rel X, const float *d_inv, const uint32_t *d_p,
                                    const uint32_t *d_q, int64_t n_pairs, float *d_out)
{
    ejoin_status s = check_pairs_args(sk, X, d_inv, d_p, d_q, nullptr, nullptr, n_pairs);
    if (s != EJOIN_OK || !d_out) return s != EJOIN_OK ? s : EJOIN_EINVAL;
    DeviceGuard g(sk->ctx->device);
    cudaStream_t st = sk->ctx->stream;
    ejoin_ctx *c = sk->ctx;
    const int64_t n = 2 * n_pairs;
    cudaError_t e;
    if ((e = grow(sk->idx, (size_t)n * 4)) || (e = grow(sk->H, (size_t)n * sk->hid * 4)) ||
        (e = grow(sk->Z, (size_t)n * sk->out * 4)) || (e = grow(sk->S, (size_t)n * sk->out * 4)))
        return from_cuda(e);
    uint32_t *idx = (uint32_t *)sk->idx.p;
    if ((e = cudaMemcpyAsync(idx, d_p, n_pairs * 4, cudaMemcpyDeviceToDevice, st)) ||
        (e = cudaMemcpyAsync(idx + n_pairs, d_q, n_pairs * 4, cudaMemcpyDeviceToDevice, st)))
        return from_cuda(e);
    float *W = P(sk->params);
    GemmArgs g1;
    g1.A = X.x;
    g1.aidx = idx;
    g1.a_rs = X.ld;
    g1.a_cs = 1;
    g1.B = W + sk->oW1;
    g1.b_rs = 1;
    g1.b_cs = sk->d;
    g1.C = P(sk->H);
    g1.ldc = sk->hid;
    g1.bias = W + sk->ob1;
    g1.rowscale = d_inv;
    g1.M = n;
    g1.N = sk->hid;
    g1.K = sk->d;
    g1.act = ACT_GELU;
    if ((e = launch_gemm_f32(g1, c->num_sms, st)) != cudaSuccess) return from_cuda(e);
    GemmArgs g2;
    g2.A = P(sk->H);
    g2.a_rs = sk->hid;
    g2.a_cs = 1;
    g2.B = W + sk->oW2;
    g2.b_rs = 1;
    g2.b_cs = sk->hid;
    g2.C = P(sk->Z);
    g2.ldc = sk->out;
    g2.bias = W + sk->ob2;
    g2.M = n;
    g2.N = sk->out;
    g2.K = sk->hid;
    if ((e = launch_gemm_f32(g2, c->num_sms, st)) != cudaSuccess) return from_cuda(e);
    if ((e = launch_rownorm(P(sk->Z), n, sk->out, P(sk->S), nullptr, c->num_sms, st)) != cudaSuccess)
        return from_cuda(e);
    return from_cuda(launch_pair_dot(P(sk->S), n_pairs, sk->out, d_out, c->num_sms, st));
}

}  // extern "C"

namespace {

constexpr int SKW = 64;
constexpr int64_t PRUNE_RECALL_ROWS = 2048;  // sampled rows of R for the recall estimate
// Threshold of the ball-row contraction: below 0 by more than its TF32 error (at most 2 * 2 * 2^-10 with the
// augmented rows' dot products bounded by 2), so that no ball pair the exact test keeps is lost.
constexpr float BALL_MARGIN = 0.006f;

// The kept tile pairs of the pruned join (sk->list, *n_list) from the balls of both sides on the tensor cores.
// cudaErrorNotSupported: the ball matrices exceed the index range of the contraction (the caller then uses the
// CUDA-core bound kernel).
cudaError_t tile_list_tc(ejoin_sketch *sk, ejoin_ctx *c, Buf &centA, Buf &radA, int64_t tA, const float *cB,
                         const float *rB, int64_t tB, float eps_sketch, bool self, unsigned long long *n_list)
{
    cudaStream_t st = c->stream;
    const int K = ball_k();
    const int64_t nbA = tA * PRUNE_BALLS, nbB = tB * PRUNE_BALLS;
    const int64_t padA = round_up(nbA, 256), padB = round_up(nbB, 256);
    if (padA >= (1ll << 31) || padB >= (1ll << 31)) return cudaErrorNotSupported;
    const uint64_t words = ((uint64_t)tA * (uint64_t)tB + 31) / 32;
    cudaError_t e;
    if ((e = ensure(sk->ballA, (size_t)padA * K * 4)) || (e = ensure(sk->ballB, (size_t)padB * K * 4)) ||
        (e = ensure(sk->bmisc, 64)) || (e = ensure(sk->bits, words * 4)) || (e = ensure(sk->rowcnt, (size_t)tA * 4)))
        return e;
    if (sk->bcand_cap == 0) sk->bcand_cap = 1ull << 22;
    long long *ncnt = (long long *)sk->bmisc.p;  // [0] ball rows of A, [1] of B
    unsigned long long *bcount = (unsigned long long *)(ncnt + 2);
    DevMisc *dm = (DevMisc *)c->misc.p;
    if ((e = launch_ball_rows(P(centA), P(radA), nbA, padA, eps_sketch, 0, P(sk->ballA), c->num_sms, st)) ||
        (e = launch_ball_rows(cB, rB, nbB, padB, eps_sketch, 1, P(sk->ballB), c->num_sms, st)) ||
        (e = launch_set_count(ncnt, nbA, st)) || (e = launch_set_count(ncnt + 1, nbB, st)))
        return e;
    CUtensorMap tmA, tmB;
    if (!make_tmap(&tmA, sk->ballA.p, FMT_F32, K, padA, 128) || !make_tmap(&tmB, sk->ballB.p, FMT_F32, K, padB, 256))
        return cudaErrorNotSupported;
    unsigned long long nb = 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
        if ((e = ensure(sk->bcand, sk->bcand_cap * sizeof(uint2))) || (e = cudaMemsetAsync(bcount, 0, 8, st)) ||
            (e = launch_sim_tc(2, &tmA, &tmB, K, ncnt, ncnt + 1, -BALL_MARGIN, nullptr, nullptr, (uint2 *)sk->bcand.p,
                               sk->bcand_cap, bcount, &dm->status, c->timeout, 0, c->num_sms, default_group_m(K), st)) ||
            (e = cudaMemcpyAsync(&nb, bcount, 8, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
            return e;
        if (nb <= sk->bcand_cap) break;
        sk->bcand_cap = nb + nb / 4 + 1024;
    }
    if (nb > sk->bcand_cap) return cudaErrorNotSupported;
    for (int attempt = 0; attempt < 3; ++attempt) {
        if ((e = ensure(sk->list, sk->list_cap * sizeof(uint2))) || (e = ensure(sk->list_count, 8)) ||
            (e = launch_ball_pairs_to_list((const uint2 *)sk->bcand.p, bcount, sk->bcand_cap, tA, tB, self ? 1 : 0,
                                           (uint32_t *)sk->bits.p, (uint32_t *)sk->rowcnt.p, (uint2 *)sk->list.p,
                                           sk->list_cap, (unsigned long long *)sk->list_count.p, c->num_sms, st)) ||
            (e = cudaMemcpyAsync(n_list, sk->list_count.p, 8, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))
            return e;
        if (*n_list <= sk->list_cap) return cudaSuccess;
        sk->list_cap = *n_list;
    }
    return cudaErrorNotSupported;
}
// covering anchors (see prune.cu): sample size, candidates per round, anchor limit, coverage cosine
constexpr int64_t COVER_SAMPLE = 262144;
constexpr int COVER_ROUND = 4096;
constexpr int COVER_MAX_ANCHORS = 32768;
constexpr float COVER_TAU = 0.85f;

// Steps 1-3 of the pruned join for one side: normalise, sketch, reorder, gather.
ejoin_status prune_side(ejoin_sketch *sk, int w, const ejoin_rel &r, int fmt, int64_t kp)
{
    ejoin_ctx *c = sk->ctx;
    cudaStream_t st = c->stream;
    auto &pw = sk->pw[w];
    Side &sd = c->side[w];
    const size_t eb = fmt_bytes(fmt);
    const int64_t n = r.n;
    const int64_t rows = round_up(std::max<int64_t>(n, 1), 256);
    const int64_t m = std::min<int64_t>(n, COVER_SAMPLE);
    cudaError_t e;
    if ((e = ensure(sd.norm, (size_t)rows * kp * eb)) || (e = ensure(sd.inv, (size_t)rows * 4)) ||
        (fmt == FMT_FP8 && (e = ensure(sd.scale, (size_t)rows * 4))) || (e = ensure(pw.S, (size_t)rows * SKW * 4)) ||
        (e = ensure(pw.key1, (size_t)rows * 4)) || (e = ensure(pw.perm, (size_t)rows * 4)) ||
        (e = ensure(pw.hist, (size_t)(COVER_MAX_ANCHORS + 1) * 4)) ||
        (e = ensure(pw.a_idx, (size_t)(m + COVER_ROUND) * 4)) || (e = ensure(pw.perm1, (size_t)COVER_ROUND)) ||
        (e = ensure(pw.anchors2, (size_t)COVER_MAX_ANCHORS * SKW * 4)) ||
        (e = ensure(pw.norm, (size_t)rows * kp * eb)) || (e = ensure(pw.inv, (size_t)rows * 4)) ||
        (fmt == FMT_FP8 && (e = ensure(pw.scale, (size_t)rows * 4))) || (e = ensure(pw.sS, (size_t)rows * SKW * 4)) ||
        (e = ensure(pw.maxdot, (size_t)std::max<int64_t>(m, 1))))
        return from_cuda(e);
    DevMisc *dm = (DevMisc *)c->misc.p;
    long long *n_dev = &dm->n_sel[w];
    if ((e = launch_set_count(n_dev, n, st)) != cudaSuccess) return from_cuda(e);
    if ((e = launch_normalize(fmt, r.x, r.ld, r.d, nullptr, n_dev, n, sd.norm.p, kp, (int)kp, (float *)sd.inv.p,
                              (float *)sd.scale.p, &dm->status, c->num_sms, st)) != cudaSuccess)
        return from_cuda(e);
    e = sketch_forward_tc(sk, r.x, n, r.ld, (const float *)sd.inv.p, (float *)pw.S.p, st);
    if (e == cudaErrorNotSupported) e = sketch_forward(sk, r.x, n, r.ld, (const float *)sd.inv.p, (float *)pw.S.p, st);
    if (e != cudaSuccess) return from_cuda(e);
    if (w == 0) cudaEventRecord(c->ev[5], st);

    // covering anchors over a strided sample of m rows, candidates taken in a fixed pseudo-random order
    const float *S = (const float *)pw.S.p;
    uint32_t *samp = (uint32_t *)pw.a_idx.p;   // sample rows [m]
    uint32_t *cand_dev = samp + m;             // this round's candidates / kept anchors
    unsigned char *drop_dev = (unsigned char *)pw.perm1.p;
    unsigned char *cov_dev = (unsigned char *)pw.maxdot.p;
    float *anchors = (float *)pw.anchors2.p;
    std::vector<uint32_t> aidx(m), order(m), cand;
    for (int64_t a = 0; a < m; ++a) aidx[a] = (uint32_t)(a * n / m), order[a] = (uint32_t)a;
    uint64_t rs = 0x9E3779B97F4A7C15ull ^ (uint64_t)(w + 1);  // splitmix64 stream for the shuffle
    auto next = [&rs]() {
        uint64_t z = (rs += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int64_t a = m - 1; a > 0; --a) std::swap(order[a], order[next() % (uint64_t)(a + 1)]);
    std::vector<unsigned char> cov(m, 0), drop(COVER_ROUND);
    if ((e = cudaMemcpyAsync(samp, aidx.data(), m * 4, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemsetAsync(cov_dev, 0, (size_t)std::max<int64_t>(m, 1), st)))
        return from_cuda(e);
    // the sample's sketches in BF16 for the coverage contraction of each round (coverage only steers the
    // reorder, so the BF16 rounding of the test is harmless)
    const int64_t rows_m = round_up(std::max<int64_t>(m, 1), 256);
    if ((e = ensure(pw.cnt, 16)) || (e = ensure(pw.smpb, (size_t)rows_m * SKW * 2)) ||
        (e = ensure(pw.rab, (size_t)COVER_ROUND * SKW * 2)))
        return from_cuda(e);
    long long *ccnt = (long long *)pw.cnt.p;
    if ((e = launch_set_count(ccnt, m, st)) ||
        (e = launch_normalize(FMT_BF16, S, SKW, SKW, samp, ccnt, m, pw.smpb.p, SKW, SKW, nullptr, nullptr, &dm->status,
                              c->num_sms, st)))
        return from_cuda(e);
    CUtensorMap tmSmp, tmRnd;
    if (!make_tmap(&tmSmp, pw.smpb.p, FMT_BF16, SKW, rows_m, 128) ||
        !make_tmap(&tmRnd, pw.rab.p, FMT_BF16, SKW, COVER_ROUND, 256))
        return EJOIN_ECUDA;
    if (c->cand_cap == 0) c->cand_cap = c->cap_hint;
    if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
    int n_anchor = 0;
    while (n_anchor < COVER_MAX_ANCHORS) {
        cand.clear();
        for (int64_t a = 0; a < m && (int)cand.size() < COVER_ROUND; ++a)
            if (!cov[order[a]]) cand.push_back(aidx[order[a]]);
        if (cand.empty()) break;
        const int nc = (int)cand.size();
        if ((e = cudaMemcpyAsync(cand_dev, cand.data(), nc * 4, cudaMemcpyHostToDevice, st)) ||
            (e = launch_cover_drop(S, cand_dev, nc, COVER_TAU, drop_dev, st)) ||
            (e = cudaMemcpyAsync(drop.data(), drop_dev, nc, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))  // cand and drop are host vectors
            return from_cuda(e);
        std::vector<uint32_t> kept;
        for (int a = 0; a < nc && n_anchor + (int)kept.size() < COVER_MAX_ANCHORS; ++a)
            if (!drop[a]) kept.push_back(cand[a]);
        const int nk = (int)kept.size();
        // the round's anchors, then the sample rows they cover: a BF16 threshold contraction of the sample
        // sketches against them on the tensor cores marks every row with cosine >= COVER_TAU to one of them
        if ((e = cudaMemcpyAsync(cand_dev, kept.data(), nk * 4, cudaMemcpyHostToDevice, st)) ||
            (e = launch_gather_rows(pw.S.p, SKW * 4, cand_dev, nk, anchors + (int64_t)n_anchor * SKW, st)) ||
            (e = launch_set_count(ccnt + 1, nk, st)) ||
            (e = launch_normalize(FMT_BF16, anchors + (int64_t)n_anchor * SKW, SKW, SKW, nullptr, ccnt + 1, nk,
                                  pw.rab.p, SKW, SKW, nullptr, nullptr, &dm->status, c->num_sms, st)))
            return from_cuda(e);
        for (int attempt = 0;; ++attempt) {
            unsigned long long n_cand = 0;
            if ((e = cudaMemsetAsync(&dm->cand_count, 0, 8, st)) ||
                (e = launch_sim_tc(0, &tmSmp, &tmRnd, SKW, ccnt, ccnt + 1, COVER_TAU, nullptr, nullptr,
                                   (uint2 *)c->cand.p, c->cand_cap, &dm->cand_count, &dm->status, c->timeout, 0,
                                   c->num_sms, default_group_m(SKW), st)) ||
                (e = launch_cover_mark((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, cov_dev, c->num_sms,
                                       st)) ||
                (e = cudaMemcpyAsync(cov.data(), cov_dev, m, cudaMemcpyDeviceToHost, st)) ||
                (e = cudaMemcpyAsync(&n_cand, &dm->cand_count, 8, cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st)))  // kept and cov are host vectors
                return from_cuda(e);
            if (n_cand <= c->cand_cap || attempt == 2) break;
            c->cand_cap = n_cand + n_cand / 4 + 1024;
            if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
        }
        n_anchor += nk;
    }
    pw.n_anchor = n_anchor;
    if (w == 0) cudaEventRecord(c->ev[6], st);

    // every row joins its most similar anchor: a BF16 threshold contraction of the sketches against
    // the anchors on the tensor cores finds, for each row, the anchors within sketch cosine 0.6, and an
    // argmax of their exact FP32 cosines picks one; rows that no anchor reaches form a last group
    const int64_t rowsK = round_up(n_anchor, 256);
    if ((e = ensure(pw.skb, (size_t)rows * SKW * 2)) || (e = ensure(pw.anb, (size_t)rowsK * SKW * 2)) ||
        (e = ensure(pw.tinv, (size_t)std::max(rows, rowsK) * 4)) || (e = ensure(pw.best, (size_t)rows * 8)) ||
        (e = ensure(pw.cnt, 16)))
        return from_cuda(e);
    long long *cnt = (long long *)pw.cnt.p;
    float *tinv = (float *)pw.tinv.p;
    if ((e = launch_set_count(cnt, n, st)) || (e = launch_set_count(cnt + 1, n_anchor, st)) ||
        (e = launch_normalize(FMT_BF16, S, SKW, SKW, nullptr, cnt, n, pw.skb.p, SKW, SKW, tinv, nullptr, &dm->status,
                              c->num_sms, st)) ||
        (e = launch_normalize(FMT_BF16, anchors, SKW, SKW, nullptr, cnt + 1, n_anchor, pw.anb.p, SKW, SKW, tinv,
                              nullptr, &dm->status, c->num_sms, st)) ||
        (e = cudaMemsetAsync(pw.best.p, 0, (size_t)n * 8, st)))
        return from_cuda(e);
    CUtensorMap tmS, tmAn;
    if (!make_tmap(&tmS, pw.skb.p, FMT_BF16, SKW, rows, 128) || !make_tmap(&tmAn, pw.anb.p, FMT_BF16, SKW, rowsK, 256))
        return EJOIN_ECUDA;
    const float thr = 0.6f - default_band(EJOIN_BF16, SKW);
    if (c->cand_cap == 0) c->cand_cap = c->cap_hint;
    if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
    for (int attempt = 0;; ++attempt) {
        DevMisc hm;
        if ((e = cudaMemsetAsync(&dm->cand_count, 0, 8, st)) ||
            (e = launch_sim_tc(0, &tmS, &tmAn, SKW, cnt, cnt + 1, thr, nullptr, nullptr, (uint2 *)c->cand.p,
                               c->cand_cap, &dm->cand_count, &dm->status, c->timeout, 0, c->num_sms,
                               default_group_m(SKW), st)) ||
            (e = cudaMemcpyAsync(&hm, dm, sizeof(DevMisc), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))
            return from_cuda(e);
        if (hm.status & ERR_TIMEOUT) return EJOIN_ETIMEOUT;
        if (hm.status & ERR_NONFINITE) return EJOIN_ENONFINITE;
        if (hm.cand_count <= c->cand_cap) break;
        if (attempt == 3) return EJOIN_ECUDA;
        c->cand_cap = hm.cand_count + hm.cand_count / 4 + 1024;
        if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
    }
    // counting sort by anchor (n_anchor + 1 groups)
    uint32_t *key = (uint32_t *)pw.key1.p, *hist = (uint32_t *)pw.hist.p, *perm = (uint32_t *)pw.perm.p;
    if ((e = launch_anchor_argmax((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, S, anchors,
                                  (unsigned long long *)pw.best.p, c->num_sms, st)) ||
        (e = launch_anchor_keys((const unsigned long long *)pw.best.p, n, n_anchor, key, c->num_sms, st)) ||
        (e = cudaMemsetAsync(hist, 0, (size_t)(n_anchor + 1) * 4, st)) || (e = launch_key_histogram(key, n, hist, st)) ||
        (e = launch_key_scan(hist, n_anchor + 1, st)) || (e = launch_key_scatter(key, n, hist, perm, st)) ||
        (e = launch_gather_rows(sd.norm.p, kp * eb, perm, n, pw.norm.p, st)) ||
        (e = launch_gather_f32((const float *)sd.inv.p, perm, n, (float *)pw.inv.p, st)) ||
        (e = launch_gather_rows(pw.S.p, SKW * 4, perm, n, pw.sS.p, st)) ||
        (fmt == FMT_FP8 && (e = launch_gather_f32((const float *)sd.scale.p, perm, n, (float *)pw.scale.p, st))))
        return from_cuda(e);
    return EJOIN_OK;
}

}  // namespace

extern "C" {

ejoin_status ejoin_threshold_pruned(ejoin_ctx *c, ejoin_sketch *sk, ejoin_rel R, ejoin_rel S, float eps,
                                    float eps_sketch, ejoin_pairs *out, ejoin_prune_stats *ps, float *recall_est)
{
    if (!c || !sk || !out || sk->ctx != c) return EJOIN_EINVAL;
    if (R.d != S.d || R.d != sk->d || R.n < 0 || S.n < 0 || R.ld < R.d || S.ld < S.d || (R.n && !R.x) ||
        (S.n && !S.x) || std::isnan(eps) || std::isnan(eps_sketch))
        return EJOIN_EINVAL;
    if (c->prec == EJOIN_F32) return EJOIN_EUNSUPPORTED;
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    c->stats = ejoin_stats{};
    ejoin_prune_stats local{};
    ejoin_prune_stats &P_ = ps ? *ps : local;
    P_ = ejoin_prune_stats{};
    out->count = 0;
    if (R.n == 0 || S.n == 0) return EJOIN_OK;
    const int fmt = fmt_of(c->prec);
    const int kind = c->prec == EJOIN_BF16 ? 0 : (c->prec == EJOIN_FP8_E4M3 ? 1 : 2);
    const int64_t kp = ejoin_padded_dim(c->prec, R.d);
    const float band = c->band_cfg >= 0.f ? c->band_cfg : default_band(c->prec, kp);
    const bool self = R.x == S.x && R.n == S.n && R.ld == S.ld;
    cudaError_t e;
    ejoin_status s;
    DevMisc *dm = (DevMisc *)c->misc.p;
    if ((e = cudaMemsetAsync(dm, 0, sizeof(DevMisc), st)) != cudaSuccess) return from_cuda(e);
    cudaEvent_t *ev = c->ev;
    cudaEventRecord(ev[0], st);
    if ((s = prune_side(sk, 0, R, fmt, kp)) != EJOIN_OK) return s;
    cudaEventRecord(ev[7], st);
    if (!self && (s = prune_side(sk, 1, S, fmt, kp)) != EJOIN_OK) return s;
    auto &pa = sk->pw[0];
    auto &pb = self ? sk->pw[0] : sk->pw[1];
    if (self && (e = launch_set_count(&dm->n_sel[1], S.n, st)) != cudaSuccess) return from_cuda(e);
    cudaEventRecord(ev[1], st);
    // tile statistics and tile-pair bounds
    const int64_t tA = (R.n + 127) / 128, tB = (S.n + 255) / 256;
    constexpr int NBL = PRUNE_BALLS;
    if ((e = ensure(pa.cent, (size_t)tA * NBL * SKW * 4)) || (e = ensure(pa.rad, (size_t)tA * NBL * 4)))
        return from_cuda(e);
    float *cB = nullptr, *rB = nullptr;
    Buf centB, radB;  // (self-join: the B side uses 256-row tiles of the same order)
    if ((e = launch_tile_stats((const float *)pa.sS.p, R.n, SKW, 128, (float *)pa.cent.p, (float *)pa.rad.p, st)) !=
        cudaSuccess)
        return from_cuda(e);
    if (self) {
        if ((e = ensure(centB, (size_t)tB * NBL * SKW * 4)) || (e = ensure(radB, (size_t)tB * NBL * 4)))
            return from_cuda(e);
        cB = (float *)centB.p;
        rB = (float *)radB.p;
    } else {
        if ((e = ensure(pb.cent, (size_t)tB * NBL * SKW * 4)) || (e = ensure(pb.rad, (size_t)tB * NBL * 4)))
            return from_cuda(e);
        cB = (float *)pb.cent.p;
        rB = (float *)pb.rad.p;
    }
    if ((e = launch_tile_stats((const float *)pb.sS.p, S.n, SKW, 256, cB, rB, st)) != cudaSuccess) {
        release(centB);
        release(radB);
        return from_cuda(e);
    }
    struct EventGuard {
        cudaEvent_t e = nullptr;
        ~EventGuard()
        {
            if (e) cudaEventDestroy(e);
        }
    } ev_stats;
    if (cudaEventCreate(&ev_stats.e) == cudaSuccess) cudaEventRecord(ev_stats.e, st);  // tile statistics done
    if (sk->list_cap == 0) sk->list_cap = std::min<uint64_t>((uint64_t)tA * tB, 1ull << 22);
    unsigned long long n_list = 0;
    // tile-pair bounds as a TF32 threshold contraction of augmented ball rows (prune.cu), the kept ball
    // pairs turned into the ordered tile list; the CUDA-core kernel below when that path cannot run
    bool listed = false;
    if ((e = tile_list_tc(sk, c, pa.cent, pa.rad, tA, cB, rB, tB, eps_sketch, self, &n_list)) == cudaSuccess)
        listed = true;
    else if (e != cudaErrorNotSupported) {
        release(centB);
        release(radB);
        return from_cuda(e);
    }
    for (int attempt = 0; attempt < 3 && !listed; ++attempt) {
        if ((e = ensure(sk->list, sk->list_cap * sizeof(uint2))) || (e = ensure(sk->list_count, 8)) ||
            (e = cudaMemsetAsync(sk->list_count.p, 0, 8, st)) ||
            (e = launch_tile_pairs((const float *)pa.cent.p, (const float *)pa.rad.p, tA, cB, rB, tB, SKW, eps_sketch,
                                   (uint2 *)sk->list.p, sk->list_cap, (unsigned long long *)sk->list_count.p, st,
                                   self ? 1 : 0)) ||
            (e = cudaMemcpyAsync(&n_list, sk->list_count.p, 8, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            release(centB);
            release(radB);
            return from_cuda(e);
        }
        if (n_list <= sk->list_cap) break;
        sk->list_cap = n_list;
    }
    if (ps) {
        // diagnostics: ball radii of both sides, covering anchors and the largest anchor group of R
        std::vector<float> ra((size_t)tA * NBL), rb((size_t)tB * NBL);
        std::vector<uint32_t> co((size_t)pa.n_anchor + 1);
        if ((e = cudaMemcpyAsync(ra.data(), pa.rad.p, ra.size() * 4, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpyAsync(rb.data(), rB, rb.size() * 4, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpyAsync(co.data(), pa.hist.p, co.size() * 4, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st))) {
            release(centB);
            release(radB);
            return from_cuda(e);
        }
        auto summarise = [](const std::vector<float> &r, float &mean, float &wide) {
            double sum = 0.0;
            uint64_t used = 0, w = 0;
            for (float x : r)
                if (x >= 0.f) {
                    sum += x;
                    ++used;
                    w += x > 0.5f;
                }
            mean = used ? (float)(sum / used) : 0.f;
            wide = used ? (float)w / (float)used : 0.f;
        };
        summarise(ra, P_.ball_radius_mean_a, P_.wide_ball_frac_a);
        summarise(rb, P_.ball_radius_mean_b, P_.wide_ball_frac_b);
        // the scatter left hist[k] at the end of anchor group k: group k holds hist[k] - hist[k - 1] rows
        uint64_t mx = 0;
        for (size_t b = 0; b < co.size(); ++b) mx = std::max<uint64_t>(mx, co[b] - (b ? co[b - 1] : 0u));
        P_.max_group_rows_a = mx;
        P_.anchors_a = (uint64_t)pa.n_anchor;
    }
    release(centB);
    release(radB);
    cudaEventRecord(ev[2], st);
    P_.tiles_total = (uint64_t)tA * tB;
    P_.tiles_kept = n_list;
    // contraction over the kept tiles
    const int64_t rowsA = round_up(R.n, 256), rowsB = round_up(S.n, 256);
    CUtensorMap tmA, tmB;
    if (!make_tmap(&tmA, pa.norm.p, fmt, kp, rowsA, 128) || !make_tmap(&tmB, pb.norm.p, fmt, kp, rowsB, 256))
        return EJOIN_ECUDA;
    if (c->cand_cap == 0) c->cand_cap = c->cap_hint;
    if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
    DevMisc hm;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((e = cudaMemsetAsync(&dm->cand_count, 0, 8, st)) ||
            (e = launch_sim_tc_list(kind, &tmA, &tmB, (int)kp, &dm->n_sel[0], &dm->n_sel[1], eps - band,
                                    (const uint2 *)sk->list.p, (const unsigned long long *)sk->list_count.p,
                                    sk->list_cap, (uint2 *)c->cand.p, c->cand_cap, &dm->cand_count, &dm->status,
                                    c->timeout, c->num_sms, st, self ? 1 : 0)) ||
            (e = cudaMemcpyAsync(&hm, dm, sizeof(DevMisc), cudaMemcpyDeviceToHost, st)) ||
            (e = cudaStreamSynchronize(st)))
            return from_cuda(e);
        if (hm.status & ERR_NONFINITE) return EJOIN_ENONFINITE;
        if (hm.status & ERR_TIMEOUT) return EJOIN_ETIMEOUT;
        if (hm.cand_count <= c->cand_cap) break;
        c->cand_cap = hm.cand_count + hm.cand_count / 4 + 1024;
        if ((e = ensure(c->cand, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
    }
    cudaEventRecord(ev[3], st);
    // result buffer and exact re-score (sorted rows map back to original ids through the permutations)
    if (out->d_pairs == nullptr) {
        void *p = nullptr;
        // a self-join writes each off-diagonal candidate in both orders
        const uint64_t cap = std::max<uint64_t>(self ? 2 * hm.cand_count : hm.cand_count, 1);
        if ((e = cudaMalloc(&p, cap * sizeof(ejoin_pair))) != cudaSuccess) return from_cuda(e);
        out->d_pairs = (ejoin_pair *)p;
        out->capacity = cap;
    }
    if (hm.cand_count) {
        if ((e = ensure(c->band, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
        // panel-ordered re-score where the rows allow it: a panel holds consecutive rows of the anchor order,
        // so its R rows are staged once in shared memory
        const bool aligned = R.d % 4 == 0 && R.d <= 1024 && R.ld % 4 == 0 && S.ld % 4 == 0 &&
                             (reinterpret_cast<uintptr_t>(R.x) & 15) == 0 && (reinterpret_cast<uintptr_t>(S.x) & 15) == 0;
        BandNorms bn;
        if (c->fp64_band > 0.f && (e = band_norms(c, R.n, S.n, &bn)) != cudaSuccess) return from_cuda(e);
        const BandNorms *bnp = c->fp64_band > 0.f ? &bn : nullptr;
        if (aligned && !(c->flags & EJOIN_FLAG_GATHER_RESCORE)) {
            if ((e = ensure(c->psorted, c->cand_cap * sizeof(uint2))) != cudaSuccess) return from_cuda(e);
            if ((e = ensure(c->pbuf, rescore_panel_buf_bytes(R.n, S.n, R.d, hm.cand_count))) != cudaSuccess)
                return from_cuda(e);
            e = launch_rescore_panels((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, (uint2 *)c->psorted.p,
                                      c->pbuf.p, R.n, S.n, hm.cand_count, &dm->n_sel[0], R.x, R.ld, S.x, S.ld, R.d,
                                      (const uint32_t *)pa.perm.p, (const uint32_t *)pb.perm.p, (const float *)pa.inv.p,
                                      (const float *)pb.inv.p, eps, c->fp64_band, out->d_pairs, out->capacity,
                                      &dm->pair_count, &dm->band_count, 0, c->num_sms, st, (uint2 *)c->band.p,
                                      c->cand_cap, self ? 1 : 0, bnp);
        } else {
            e = launch_rescore((const uint2 *)c->cand.p, &dm->cand_count, c->cand_cap, R.x, R.ld, S.x, S.ld, R.d,
                               (const uint32_t *)pa.perm.p, (const uint32_t *)pb.perm.p, (const float *)pa.inv.p,
                               (const float *)pb.inv.p, eps, c->fp64_band, out->d_pairs, out->capacity,
                               &dm->pair_count, &dm->band_count, 0, c->num_sms, st, (uint2 *)c->band.p, c->cand_cap,
                               self ? 1 : 0, bnp);
        }
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (out->d_count &&
        (e = cudaMemcpyAsync(out->d_count, &dm->pair_count, 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return from_cuda(e);
    cudaEventRecord(ev[4], st);
    if ((e = cudaMemcpyAsync(&hm, dm, sizeof(DevMisc), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return from_cuda(e);
    auto ms = [&](int a, int b) {
        float x = 0.f;
        cudaEventElapsedTime(&x, ev[a], ev[b]);
        return x;
    };
    P_.candidates = hm.cand_count;
    P_.pairs = hm.pair_count;
    P_.ms_prepare = ms(0, 1);
    P_.ms_bound = ms(1, 2);
    if (ev_stats.e) {
        float x = 0.f;
        cudaEventElapsedTime(&x, ev[1], ev_stats.e);
        P_.ms_tile_stats = x;
    }
    P_.ms_contract = ms(2, 3);
    P_.ms_rescore = ms(3, 4);
    P_.ms_total = ms(0, 4);
    P_.ms_sketch_a = ms(0, 5);
    P_.ms_cover_a = ms(5, 6);
    P_.ms_assign_a = ms(6, 7);
    c->stats.candidates = hm.cand_count;
    c->stats.pairs = hm.pair_count;
    c->stats.fp64_rescored = hm.band_count;
    c->stats.band = band;
    out->count = hm.pair_count;
    if (recall_est) {
        // recall estimate: the exact join of every stride-th row of R with S (the plain path), and the share
        // of its matches whose tile pair the pruned join kept (each such match is found: its bulk
        // similarity is within the band, and the re-score decides it as the plain join does)
        const ejoin_stats pruned_stats = c->stats;
        const int64_t m = std::min<int64_t>(R.n, PRUNE_RECALL_ROWS);
        const int64_t stride = R.n / m;
        const ejoin_rel Rs{R.x, m, R.d, R.ld * stride};
        const uint32_t flags0 = c->flags;
        c->flags &= ~(EJOIN_FLAG_SORT | EJOIN_FLAG_COUNT_ONLY | EJOIN_FLAG_FUSED);
        ejoin_pairs sp{nullptr, 0, nullptr, 0};
        s = ejoin_threshold(c, Rs, S, eps, nullptr, nullptr, &sp);
        c->flags = flags0;
        c->stats = pruned_stats;
        Buf scr;
        const size_t sb = recall_probe_scratch_bytes(R.n, S.n, tA, tB);
        unsigned long long found = 0;
        if (s == EJOIN_OK) {
            if ((e = ensure(scr, sb + 8)) ||
                (e = launch_recall_probe((const uint32_t *)pa.perm.p, R.n, (const uint32_t *)pb.perm.p, S.n,
                                         (const uint2 *)sk->list.p, (const unsigned long long *)sk->list_count.p,
                                         sk->list_cap, tA, tB, sp.d_pairs, sp.count, (uint32_t)stride, self ? 1 : 0,
                                         scr.p, (unsigned long long *)((char *)scr.p + sb), c->num_sms, st)) ||
                (e = cudaMemcpyAsync(&found, (char *)scr.p + sb, 8, cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st)))
                s = from_cuda(e);
        }
        release(scr);
        const uint64_t total = sp.count;
        ejoin_pairs_free(c, &sp);
        if (s != EJOIN_OK) return s;
        P_.recall_est = total ? (float)((double)found / (double)total) : 1.f;
        P_.recall_sample_rows = (uint64_t)m;
        P_.recall_sample_matches = total;
        *recall_est = P_.recall_est;
    }
    if (hm.pair_count > out->capacity) return EJOIN_EOVERFLOW;
    if (c->flags & EJOIN_FLAG_SORT) return sort_result(c, out->d_pairs, hm.pair_count, R.n, S.n);
    return EJOIN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------------------
// Training of the sketch network with its labelled set and calibration (ejoin_sketch_train).
namespace {

// Records of a sorted join as separate row arrays: p[k] = pairs[k].i, q[k] = pairs[k].j.
cudaError_t split_pairs(const ejoin_pair *pairs, uint64_t n, uint32_t *p, uint32_t *q, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpy2DAsync(p, 4, &pairs[0].i, sizeof(ejoin_pair), 4, n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(q, 4, &pairs[0].j, sizeof(ejoin_pair), 4, n, cudaMemcpyDeviceToDevice, st);
    return e;
}

// The exact self-join of X at eps, sorted by (i, j), into a library-allocated buffer (caller frees it).
ejoin_status sorted_self_join(ejoin_ctx *c, const ejoin_rel &X, float eps, ejoin_pairs *out)
{
    const uint32_t flags0 = c->flags;
    c->flags = (flags0 | EJOIN_FLAG_SORT) & ~(EJOIN_FLAG_COUNT_ONLY | EJOIN_FLAG_FUSED);
    *out = ejoin_pairs{nullptr, 0, nullptr, 0};
    const ejoin_status s = ejoin_threshold(c, X, X, eps, nullptr, nullptr, out);
    c->flags = flags0;
    return s;
}

bool rel_valid(const ejoin_rel &X, int d) { return X.x && X.d == d && X.ld >= X.d && X.n >= 2 && X.n < (1ll << 31); }

}  // namespace

extern "C" {

ejoin_status ejoin_sketch_train(ejoin_sketch *sk, ejoin_rel X_train, ejoin_rel X_cal,
                                const ejoin_sketch_train_cfg *cfg_in, float *eps_sketch,
                                ejoin_sketch_train_report *report)
{
    if (!sk || !cfg_in || !eps_sketch || !rel_valid(X_train, sk->d) || !rel_valid(X_cal, sk->d)) return EJOIN_EINVAL;
    ejoin_sketch_train_cfg cfg = *cfg_in;
    if (!(cfg.eps == cfg.eps)) return EJOIN_EINVAL;
    if (cfg.label_margin <= 0.f) cfg.label_margin = 0.2f;
    if (cfg.w_join <= 0.f) cfg.w_join = 8.f;
    if (cfg.n_pairs <= 0) cfg.n_pairs = 10000000;
    if (cfg.epochs <= 0) cfg.epochs = 3;
    if (cfg.batch <= 0) cfg.batch = 65536;
    if (cfg.lr <= 0.f) cfg.lr = 2e-3f;
    if (cfg.recall <= 0.f || cfg.recall > 1.f) cfg.recall = 0.999f;
    if (cfg.cal_margin < 0.f) cfg.cal_margin = 0.01f;
    if (cfg.n_pairs > (1ll << 31) || cfg.batch > (1 << 24)) return EJOIN_EINVAL;
    ejoin_ctx *c = sk->ctx;
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    ejoin_sketch_train_report rep{};
    cudaError_t e = cudaSuccess;
    ejoin_status s = EJOIN_OK;
    Buf lab, scratch, inv, batch, cal, rec;
    ejoin_pairs jp{nullptr, 0, nullptr, 0};
    cudaEvent_t ev[4] = {};
    auto done = [&](ejoin_status r) {
        if (jp.d_pairs) ejoin_pairs_free(c, &jp);
        cudaStreamSynchronize(st);
        for (Buf *b : {&lab, &scratch, &inv, &batch, &cal, &rec}) release(*b);
        for (auto &x : ev)
            if (x) cudaEventDestroy(x);
        return r;
    };
    for (auto &x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) return done(EJOIN_ECUDA);
    const uint64_t seed = cfg.seed;
    cudaEventRecord(ev[0], st);
    if (cfg.init) {
        const size_t bytes = (size_t)sk->n_params * 4;
        if ((e = launch_init_params(P(sk->params), sk->d, sk->hid, sk->out, seed, c->num_sms, st)) ||
            (e = cudaMemsetAsync(sk->m.p, 0, bytes, st)) || (e = cudaMemsetAsync(sk->v.p, 0, bytes, st)))
            return done(from_cuda(e));
        sk->step = 0;
    }

    // 1. labelled set: the exact self-join of the training sample at eps - label_margin (matches and near
    //    misses, each with its exact similarity as target), subsampled to about half of n_pairs, then
    //    uniform random pairs scored exactly
    if ((s = sorted_self_join(c, X_train, cfg.eps - cfg.label_margin, &jp)) != EJOIN_OK) return done(s);
    rep.label_join_pairs = jp.count;
    const int64_t n_pairs = cfg.n_pairs;
    const uint64_t off_diag = jp.count > (uint64_t)X_train.n ? jp.count - (uint64_t)X_train.n : 1;
    const double frac = std::min(1.0, (double)(n_pairs / 2) / (double)off_diag);
    const uint32_t keep = frac >= 1.0 ? 0xffffffffu : (uint32_t)(frac * 4294967296.0);
    const uint64_t cap = (uint64_t)n_pairs;  // join pairs first, random pairs fill the rest
    uint32_t *lp, *lq;
    float *lt, *lw;
    if ((e = ensure(lab, (size_t)cap * 16)) ||
        (e = ensure(scratch, label_scratch_bytes(jp.count) + 64)) ||
        (e = ensure(inv, (size_t)X_train.n * 4)))
        return done(from_cuda(e));
    lp = (uint32_t *)lab.p;
    lq = lp + cap;
    lt = (float *)(lq + cap);
    lw = lt + cap;
    unsigned long long *d_total = (unsigned long long *)((char *)scratch.p + label_scratch_bytes(jp.count));
    // the draw keeps about n_pairs / 2 of the join pairs (at most cap are written)
    if ((e = launch_label_join_pairs(jp.d_pairs, jp.count, seed, keep, cfg.w_join, scratch.p, d_total, cap, lp, lq,
                                     lt, lw, st)))
        return done(from_cuda(e));
    unsigned long long kept = 0;
    if ((e = cudaMemcpyAsync(&kept, d_total, 8, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
        return done(from_cuda(e));
    ejoin_pairs_free(c, &jp);
    jp = ejoin_pairs{nullptr, 0, nullptr, 0};
    kept = std::min<unsigned long long>(kept, (unsigned long long)n_pairs);
    const int64_t n_rand = n_pairs - (int64_t)kept;
    if ((e = launch_row_inv_norm(X_train.x, X_train.n, X_train.d, X_train.ld, (float *)inv.p, c->num_sms, st)) ||
        (e = launch_random_pairs(lp + kept, lq + kept, lw + kept, n_rand, (uint32_t)X_train.n, seed, c->num_sms,
                                 st)) ||
        (e = launch_score_pairs(X_train.x, X_train.ld, X_train.x, X_train.ld, X_train.d, lp + kept, lq + kept,
                                (const float *)inv.p, (const float *)inv.p, n_rand, lt + kept, c->num_sms, st)))
        return done(from_cuda(e));
    rep.labelled_join = kept;
    rep.labelled_random = (uint64_t)n_rand;
    cudaEventRecord(ev[1], st);

    // 2. epochs of Adam steps over the labelled set, in a seeded order per epoch
    const int64_t n_lab = (int64_t)kept + n_rand;
    const int64_t bsz = std::min<int64_t>(cfg.batch, n_lab);
    if ((e = ensure(batch, (size_t)bsz * 16))) return done(from_cuda(e));
    uint32_t *bp = (uint32_t *)batch.p, *bq = bp + bsz;
    float *bt = (float *)(bq + bsz), *bw = bt + bsz;
    bool first = true;
    for (int ep = 0; ep < cfg.epochs; ++ep) {
        for (int64_t b0 = 0; b0 < n_lab; b0 += bsz) {
            const int64_t m = std::min<int64_t>(bsz, n_lab - b0);
            if ((e = launch_gather_batch(lp, lq, lt, lw, (uint64_t)n_lab, seed, ep, (uint64_t)b0, m, bp, bq, bt, bw,
                                         c->num_sms, st)) ||
                (e = sketch_grad(sk, X_train.x, X_train.ld, (const float *)inv.p, bp, bq, bt, bw, m, st)))
                return done(from_cuda(e));
            sk->step += 1;
            if ((e = launch_adam(P(sk->params), P(sk->grads), P(sk->m), P(sk->v), sk->n_params, cfg.lr, 0.9f, 0.999f,
                                 1e-8f, sk->step, c->num_sms, st)))
                return done(from_cuda(e));
            const bool last = ep == cfg.epochs - 1 && b0 + bsz >= n_lab;
            if (first || last) {
                float loss = 0.f;  // the loss of this step's batch, before its update
                if ((e = cudaMemcpyAsync(&loss, sk->scal.p, 4, cudaMemcpyDeviceToHost, st)) ||
                    (e = cudaStreamSynchronize(st)))
                    return done(from_cuda(e));
                if (first) rep.loss_first = loss;
                if (last) rep.loss_last = loss;
                first = false;
            }
        }
    }
    cudaEventRecord(ev[2], st);

    // 3. calibration: eps_sketch is the (1 - recall) quantile of the sketch cosine over the exact matches
    //    of the calibration sample (linear interpolation between order statistics), less cal_margin
    if ((s = sorted_self_join(c, X_cal, cfg.eps, &jp)) != EJOIN_OK) return done(s);
    const uint64_t nm = jp.count;
    rep.calibration_matches = nm;
    float eps_sk = -1.f;
    if (nm > 0) {
        if ((e = ensure(cal, (size_t)nm * 12 + (size_t)X_cal.n * 4)) ||
            (e = ensure(rec, (size_t)nm * 2 * sizeof(ejoin_pair) + sort_pairs_scratch_bytes(nm))))
            return done(from_cuda(e));
        uint32_t *cp = (uint32_t *)cal.p, *cq = cp + nm;
        float *cs = (float *)(cq + nm), *cinv = cs + nm;
        ejoin_pair *r0 = (ejoin_pair *)rec.p, *r1 = r0 + nm;
        void *sscr = r1 + nm;
        if ((e = split_pairs(jp.d_pairs, nm, cp, cq, st)) ||
            (e = launch_row_inv_norm(X_cal.x, X_cal.n, X_cal.d, X_cal.ld, cinv, c->num_sms, st)))
            return done(from_cuda(e));
        if ((s = ejoin_sketch_pair_sims(sk, X_cal, cinv, cp, cq, (int64_t)nm, cs)) != EJOIN_OK) return done(s);
        if ((e = launch_value_records(cs, (int64_t)nm, r0, c->num_sms, st)) ||
            (e = launch_sort_pairs(r0, r1, nm, 1ull << 32, nm, sscr, st)))
            return done(from_cuda(e));
        const double pos = (1.0 - (double)cfg.recall) * (double)(nm - 1);
        const uint64_t lo = (uint64_t)pos;
        const uint64_t hi = std::min<uint64_t>(lo + 1, nm - 1);
        ejoin_pair a{}, b{};
        if ((e = cudaMemcpyAsync(&a, r0 + lo, sizeof a, cudaMemcpyDeviceToHost, st)) ||
            (e = cudaMemcpyAsync(&b, r0 + hi, sizeof b, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
            return done(from_cuda(e));
        const double q = (double)a.sim + ((double)b.sim - (double)a.sim) * (pos - (double)lo);
        eps_sk = (float)(q - (double)cfg.cal_margin);
    }
    cudaEventRecord(ev[3], st);
    if ((e = cudaStreamSynchronize(st))) return done(from_cuda(e));
    cudaEventElapsedTime(&rep.ms_label, ev[0], ev[1]);
    cudaEventElapsedTime(&rep.ms_train, ev[1], ev[2]);
    cudaEventElapsedTime(&rep.ms_calibrate, ev[2], ev[3]);
    rep.eps_sketch = eps_sk;
    *eps_sketch = eps_sk;
    if (report) *report = rep;
    return done(EJOIN_OK);
}

}  // extern "C"
