// LSQR as iterative regularization (Sec. 3.4) on a finished GKB run.
//
// The k-th LSQR iterate is x_k = Z_k y_k with y_k the least-squares solution
// of C_k y = beta_1 e_1.  Because C_k is lower bidiagonal and the C_k are
// nested, one sweep of Givens rotations (the bidiagonal QR of Paige and
// Saunders' LSQR) serves every k:
//   rb_1 = alpha_1, pb_1 = beta_1;  for i = 1..l:
//     d_i = |(rb_i, beta_{i+1})|, c_i = rb_i / d_i, s_i = beta_{i+1} / d_i,
//     th_{i+1} = s_i alpha_{i+1}, rb_{i+1} = -c_i alpha_{i+1},
//     ph_i = c_i pb_i, pb_{i+1} = s_i pb_i,
// so that R_k y_k = (ph_1..ph_k) with R_k upper bidiagonal (d on the
// diagonal, th above), and |A x_k - f| = |C_k y_k - beta_1 e_1| = |pb_{k+1}|.
// eta_k = |x_k| = |y_k| (Z_k orthonormal) needs each y_k: one thread per k
// back-substitutes.  The stopping index follows the L-curve corner of
// (ln rho_k, ln eta_k) (curvature by central differences along decreasing k)
// or the projected GCV rho_k^2 / ((l+1) - k)^2; then x_k = Z_k y_k.
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int LQ_T = 512;
constexpr int LQ_MAX = 511;  // steps handled (shared-memory sequences)

// One block.  rule 0 GCV, 1 L-curve, 2 fixed k.
__global__ void __launch_bounds__(LQ_T) k_lsqr(const double* __restrict__ alpha, const double* __restrict__ beta,
                                               int l, int rule, int k_fixed, double* __restrict__ y_out,
                                               double* __restrict__ curve, rbf_dev_state* __restrict__ stt) {
    __shared__ double d_inv[LQ_MAX], th[LQ_MAX + 1], ph[LQ_MAX], rho[LQ_MAX], leta[LQ_MAX], lrho[LQ_MAX];
    __shared__ double bv[LQ_T];
    __shared__ int bi[LQ_T];
    if (threadIdx.x == 0) {
        double rb = alpha[0], pb = beta[0];
        for (int i = 1; i <= l; ++i) {
            const double b = beta[i];  // beta_{i+1}
            const double q = fma(rb, rb, b * b);
            const double inv = rsqrt_f64(q);
            const double c = rb * inv, s = b * inv;
            d_inv[i - 1] = inv;
            ph[i - 1] = c * pb;
            pb = s * pb;
            rho[i - 1] = fabs(pb);
            if (i < l) {
                th[i] = s * alpha[i];
                rb = -c * alpha[i];
            }
        }
    }
    __syncthreads();
    // eta_k by back substitution, one thread per k
    for (int k = threadIdx.x + 1; k <= l; k += LQ_T) {
        double y = ph[k - 1] * d_inv[k - 1];
        double e2 = y * y;
        for (int i = k - 1; i >= 1; --i) {
            y = (ph[i - 1] - th[i] * y) * d_inv[i - 1];
            e2 = fma(y, y, e2);
        }
        leta[k - 1] = 0.5 * log(e2);
        lrho[k - 1] = log(rho[k - 1]);
    }
    __syncthreads();
    double best = rule == 1 ? -INFINITY : INFINITY;
    int besti = 0x7fffffff;
    if (rule != 2) {
        for (int k = threadIdx.x + 1; k <= l; k += LQ_T) {
            double v;
            if (rule == 0) {
                const double dd = (double)(l + 1 - k);
                v = rho[k - 1] * rho[k - 1] / (dd * dd);
                if (curve) curve[k - 1] = v;
                if (isnan(v)) v = INFINITY;
                if (v < best || (v == best && k < besti)) { best = v; besti = k; }
            } else {
                v = -INFINITY;
                if (k >= 2 && k <= l - 1) {
                    // derivatives along decreasing k (growing regularization)
                    const double x1 = 0.5 * (lrho[k - 2] - lrho[k]), y1 = 0.5 * (leta[k - 2] - leta[k]);
                    const double x2 = lrho[k] - 2.0 * lrho[k - 1] + lrho[k - 2];
                    const double y2 = leta[k] - 2.0 * leta[k - 1] + leta[k - 2];
                    const double sp = x1 * x1 + y1 * y1;
                    v = (x1 * y2 - x2 * y1) / (sp * sqrt(sp));
                    if (!isfinite(v) || !(sp >= 1e-8)) v = -INFINITY;
                }
                if (curve) curve[k - 1] = v;
                if (v > best || (v == best && k < besti)) { best = v; besti = k; }
            }
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int off = LQ_T / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            const double ov = bv[threadIdx.x + off], mv = bv[threadIdx.x];
            const int oi = bi[threadIdx.x + off], mi = bi[threadIdx.x];
            const bool take = rule == 1 ? (ov > mv || (ov == mv && oi < mi)) : (ov < mv || (ov == mv && oi < mi));
            if (take) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int k = rule == 2 ? k_fixed : bi[0];
        if (k < 1 || k > l) k = l;  // no finite candidate: the last iterate
        double y = ph[k - 1] * d_inv[k - 1];
        double e2 = y * y;
        y_out[k - 1] = y;
        for (int i = k - 1; i >= 1; --i) {
            y = (ph[i - 1] - th[i] * y) * d_inv[i - 1];
            y_out[i - 1] = y;
            e2 = fma(y, y, e2);
        }
        stt->info[IN_RANK] = k;
        stt->info[IN_INDEX] = -1;
        stt->scal[SC_LAMBDA] = 0.0;
        stt->scal[SC_ETA] = sqrt(e2);
        stt->scal[SC_RHO] = rho[k - 1];
    }
}

// coef = Z_k y (one thread per row, Z column-major with ld ldz)
__global__ void k_lsqr_lift(const double* __restrict__ Z, int64_t ldz, int64_t n, const rbf_dev_state* __restrict__ stt,
                            const double* __restrict__ y, double* __restrict__ coef) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = stt->info[IN_RANK];
    double acc = 0.0;
    for (int m = 0; m < k; ++m) acc = fma(Z[(int64_t)m * ldz + i], y[m], acc);
    coef[i] = acc;
}

}  // namespace

extern "C" rbf_status rbf_lsqr(rbf_ctx* ctx, const rbf_gkb_state* st, int rule, int k_fixed, double* d_coef,
                               double* d_curve, rbf_solve_info* info) {
    RbfRange range_("rbf_lsqr");
    if (!ctx) return RBF_ERR_INVALID;
    if (!st || !d_coef) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_lsqr: NULL argument");
    const int l = st->steps_done;
    if (l < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "state has no completed step");
    if (l > LQ_MAX) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "more than %d steps", LQ_MAX);
    if (rule != RBF_GCV && rule != RBF_LCURVE && rule != RBF_FIXED)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rule must be RBF_GCV, RBF_LCURVE or RBF_FIXED");
    if (rule == RBF_FIXED && (k_fixed < 1 || k_fixed > l))
        return rbf_fail(ctx, RBF_ERR_INVALID, "k = %d outside [1, l = %d]", k_fixed, l);
    RBF_TRY(rbf_ws_reserve(ctx, ws_align((size_t)l * 8)));
    double* y = (double*)ctx->ws;
    k_lsqr<<<1, LQ_T, 0, ctx->stream>>>(st->d_alpha, st->d_beta, l, rule, k_fixed, y, d_curve, ctx->d_state);
    RBF_LAUNCHED(ctx, "k_lsqr");
    k_lsqr_lift<<<(unsigned)((st->n + 255) / 256), 256, 0, ctx->stream>>>(st->d_Z, st->ldz, st->n, ctx->d_state, y,
                                                                          d_coef);
    RBF_LAUNCHED(ctx, "k_lsqr_lift");
    RBF_CUDA(ctx, cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(rbf_dev_state), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RBF_CUDA(ctx, cudaGetLastError());
    if (info) {
        info->lambda = 0.0;
        info->index = -1;
        info->rank = ctx->h_state->info[IN_RANK];
        info->steps = l;
        info->sigma1 = 0.0;
        info->eta = ctx->h_state->scal[SC_ETA];
        info->rho = ctx->h_state->scal[SC_RHO];
    }
    return RBF_OK;
}
