// Parameter choice and projected solves (Algorithms 2 and 4), lift alpha = Z_l y.
//
// Grid: lambda_t = s~_1 10^{t}, t = t_lo + (t_hi - t_lo) * idx / (J - 1).
// For each grid point (one thread each):
//   q_i = lambda^2 / (s~_i^2 + lambda^2)         (= 1 - phi~_i)
//   rho^2 = sum_i q_i^2 f~_i^2 + f~_{l+1}^2         (eq. rho_proj)
//   eta^2 = sum_i (s~_i f~_i / (s~_i^2 + lambda^2))^2 (eq. eta_proj)
//   GCV   = rho^2 / (1 + sum_i q_i)^2                (eq. gcv_proj: (l+1) - sum phi~_i)
// GCV: grid argmin, smallest index on ties.  L-curve: signed curvature of
// (ln rho, ln eta) by central differences in t at interior points, argmax over
// the points whose speed is at least 1e-4 per decade (stationary stretches of
// the curve carry only rounding noise).
// HKT: y = V~ (s~_i f~_i / (s~_i^2 + lambda^2))_i (the SVD form of the normal
// equations of Algorithm 4 step 9).  Ine-TSVD: GCV_l(k) = (sum_{i>k} f~_i^2 +
// f~_{l+1}^2) / ((l+1) - k)^2 over k = 1..r_l, r_l = #{s~_i > (l+1) eps s~_1};
// y = V~ (f~_i / s~_i for i <= k).
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace {

__device__ __forceinline__ int sel_l(const ProjDims& d, int b) { return d.l_arr ? d.l_arr[b] : d.l; }

__global__ void k_grid_terms(ProjDims d, const double* __restrict__ sigma_all, const double* __restrict__ ftil_all,
                             int J, double t_lo, double t_hi, double* __restrict__ gcv_all,
                             double* __restrict__ xr_all, double* __restrict__ ye_all) {
    const int b = blockIdx.y;
    const int l = sel_l(d, b);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= J || l < 1) return;
    const double* sigma = sigma_all + (size_t)b * d.L;
    const double* ftil = ftil_all + (size_t)b * (d.L + 1);
    const double lam = sigma[0] * exp10(grid_t(t, J, t_lo, t_hi));
    const double lam2 = lam * lam;
    double rho2 = 0.0, eta2 = 0.0, den = 1.0;
    for (int i = 0; i < l; ++i) {
        const double s = sigma[i], f = ftil[i];
        const double inv = 1.0 / fma(s, s, lam2);
        const double q = lam2 * inv;
        const double g = s * f * inv;
        rho2 = fma(q * q, f * f, rho2);
        eta2 = fma(g, g, eta2);
        den += q;
    }
    rho2 = fma(ftil[l], ftil[l], rho2);
    gcv_all[(size_t)b * J + t] = rho2 / (den * den);
    xr_all[(size_t)b * J + t] = 0.5 * log(rho2);
    ye_all[(size_t)b * J + t] = 0.5 * log(eta2);
}

// Choose lambda (rule 0 GCV, 1 L-curve, 2 fixed, 3 fixed t: lambda = s~_1
// 10^lambda_in) and form the coefficient vector cvec_i = s_i f_i / (s_i^2 +
// lambda^2); eta = |cvec| and rho (eq. rho_proj) at that lambda go to the
// state (instance 0).  One block per instance.
__global__ void k_choose_lambda(ProjDims d, const double* __restrict__ sigma_all,
                                const double* __restrict__ ftil_all, int J, double t_lo, double t_hi,
                                int rule0, double lambda0, const int* __restrict__ rule_arr,
                                const double* __restrict__ lam_arr, const double* __restrict__ gcv_all,
                                const double* __restrict__ xr_all, const double* __restrict__ ye_all,
                                double* __restrict__ curve_all, double* __restrict__ cvec_all,
                                double* __restrict__ lam_out, int* __restrict__ idx_out,
                                rbf_dev_state* __restrict__ stt) {
    __shared__ double bv[1024];
    __shared__ double gcv_red[1024];
    __shared__ int bi[1024];
    __shared__ double lam_s;
    const int b = blockIdx.x;
    const int l = sel_l(d, b);
    if (l < 1) return;
    const int rule = rule_arr ? rule_arr[b] : rule0;  // per-instance rule and lambda_in when given
    const double lambda_in = lam_arr ? lam_arr[b] : lambda0;
    const double* sigma = sigma_all + (size_t)b * d.L;
    const double* ftil = ftil_all + (size_t)b * (d.L + 1);
    const double* gcv = gcv_all + (size_t)b * J;
    const double* xr = xr_all + (size_t)b * J;
    const double* ye = ye_all + (size_t)b * J;
    double* curve = curve_all ? curve_all + (size_t)b * J : nullptr;
    double* cvec = cvec_all + (size_t)b * d.L;
    const double h = (t_hi - t_lo) / (double)(J - 1);
    // per-thread best over a strided subset, then a tree with lowest-index tie-break
    double best = rule == 1 ? -INFINITY : INFINITY;
    int besti = 0x7fffffff;
    if (rule < 2) {
        for (int t = threadIdx.x; t < J; t += blockDim.x) {
            double v;
            if (rule == 0) {
                v = gcv[t];
                if (curve) curve[t] = v;
                if (isnan(v)) v = INFINITY;
                if (v < best || (v == best && t < besti)) { best = v; besti = t; }
            } else {
                v = -INFINITY;
                if (t > 0 && t < J - 1) {
                    const double x1 = (xr[t + 1] - xr[t - 1]) / (2.0 * h);
                    const double y1 = (ye[t + 1] - ye[t - 1]) / (2.0 * h);
                    const double x2 = (xr[t + 1] - 2.0 * xr[t] + xr[t - 1]) / (h * h);
                    const double y2 = (ye[t + 1] - 2.0 * ye[t] + ye[t - 1]) / (h * h);
                    const double sp = x1 * x1 + y1 * y1;
                    v = (x1 * y2 - x2 * y1) / (sp * sqrt(sp));
                    // stationary points (speed < 1e-4 per decade) are not candidates
                    if (!isfinite(v) || !(sp >= 1e-8)) v = -INFINITY;
                }
                if (curve) curve[t] = v;
                if (v > best || (v == best && t < besti)) { best = v; besti = t; }
            }
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            const double ov = bv[threadIdx.x + off];
            const int oi = bi[threadIdx.x + off];
            const double mv = bv[threadIdx.x];
            const int mi = bi[threadIdx.x];
            const bool take = rule == 1 ? (ov > mv || (ov == mv && oi < mi)) : (ov < mv || (ov == mv && oi < mi));
            if (take) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double lam;
        int idx;
        if (rule == 2) {
            lam = lambda_in;
            idx = -1;
        } else if (rule == 3) {
            lam = sigma[0] * exp10(lambda_in);
            idx = -1;
        } else {
            idx = bi[0];
            if (idx < 0 || idx >= J) idx = 0;
            lam = sigma[0] * exp10(grid_t(idx, J, t_lo, t_hi));
        }
        lam_s = lam;
        if (lam_out) lam_out[b] = lam;
        if (idx_out) idx_out[b] = idx;
        if (stt && b == 0) {
            stt->scal[SC_LAMBDA] = lam;
            stt->scal[SC_SIGMA1] = sigma[0];
            stt->info[IN_INDEX] = idx;
        }
    }
    __syncthreads();
    const double lam2 = lam_s * lam_s;
    double e2 = 0.0, r2 = 0.0;
    for (int i = threadIdx.x; i < l; i += blockDim.x) {
        const double s = sigma[i];
        const double inv = 1.0 / fma(s, s, lam2);
        const double cv = s * ftil[i] * inv;
        const double q = lam2 * inv * ftil[i];
        cvec[i] = cv;
        e2 = fma(cv, cv, e2);
        r2 = fma(q, q, r2);
    }
    if (stt && b == 0) {
        __syncthreads();
        bv[threadIdx.x] = e2;
        gcv_red[threadIdx.x] = r2;
        __syncthreads();
        for (int off = blockDim.x / 2; off > 0; off >>= 1) {
            if ((int)threadIdx.x < off) {
                bv[threadIdx.x] += bv[threadIdx.x + off];
                gcv_red[threadIdx.x] += gcv_red[threadIdx.x + off];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            stt->scal[SC_ETA] = sqrt(bv[0]);
            stt->scal[SC_RHO] = sqrt(fma(ftil[l], ftil[l], gcv_red[0]));
        }
    }
}

// Ine-TSVD rank by GCV_l(k) (or the given rank) and cvec_i = f_i / s_i, i <= k.
__global__ void k_choose_rank(ProjDims d, const double* __restrict__ sigma_all,
                              const double* __restrict__ ftil_all, int rank_in, double* __restrict__ curve_all,
                              double* __restrict__ cvec_all, double* __restrict__ work_all,
                              int* __restrict__ rank_out, rbf_dev_state* __restrict__ stt) {
    __shared__ int k_s;
    const int b = blockIdx.x;
    const int l = sel_l(d, b);
    if (l < 1) return;
    const double* sigma = sigma_all + (size_t)b * d.L;
    const double* ftil = ftil_all + (size_t)b * (d.L + 1);
    double* curve = curve_all ? curve_all + (size_t)b * d.L : nullptr;
    double* cvec = cvec_all + (size_t)b * d.L;
    double* work = work_all + (size_t)b * (d.L + 2);
    if (threadIdx.x == 0) {
        const double s1 = sigma[0];
        int r = 0;
        for (int i = 0; i < l; ++i) r += sigma[i] > (double)(l + 1) * DBL_EPSILON * s1 ? 1 : 0;
        int k = rank_in;
        if (k <= 0) {
            // suffix sums S_k = sum_{i=k+1}^{l} f_i^2 + f_{l+1}^2 (1-based i), k = l..1
            double acc = ftil[l] * ftil[l];
            for (int kk = l; kk >= 1; --kk) {
                work[kk] = acc;       // S_kk
                acc = fma(ftil[kk - 1], ftil[kk - 1], acc);
            }
            double best = INFINITY;
            k = 1;
            for (int kk = 1; kk <= r; ++kk) {
                const double dd = (double)(l + 1 - kk);
                const double gv = work[kk] / (dd * dd);
                if (curve) curve[kk - 1] = gv;
                if (gv < best) {
                    best = gv;
                    k = kk;
                }
            }
            if (r == 0) k = 1;
        }
        if (k > l) k = l;
        k_s = k;
        if (rank_out) rank_out[b] = k;
        if (stt && b == 0) {
            double e2 = 0.0, r2 = ftil[l] * ftil[l];
            for (int i = 0; i < l; ++i) {
                if (i < k) {
                    const double cv = ftil[i] / sigma[i];
                    e2 = fma(cv, cv, e2);
                } else {
                    r2 = fma(ftil[i], ftil[i], r2);
                }
            }
            stt->info[IN_RANK] = k;
            stt->scal[SC_SIGMA1] = s1;
            stt->scal[SC_ETA] = sqrt(e2);
            stt->scal[SC_RHO] = sqrt(r2);
        }
    }
    __syncthreads();
    const int k = k_s;
    for (int i = threadIdx.x; i < l; i += blockDim.x) cvec[i] = i < k ? ftil[i] / sigma[i] : 0.0;
}

// y = V cvec (V column-major l x l, ld ldv), per instance
__global__ void k_vmul(ProjDims d, const double* __restrict__ V_all, int64_t ldv,
                       const double* __restrict__ cvec_all, double* __restrict__ y_all) {
    const int b = blockIdx.y;
    const int l = sel_l(d, b);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= l) return;
    const double* V = V_all + (size_t)b * d.L * ldv;
    const double* cvec = cvec_all + (size_t)b * d.L;
    double acc = 0.0;
    for (int i = 0; i < l; ++i) acc = fma(V[(int64_t)i * ldv + r], cvec[i], acc);
    y_all[(size_t)b * d.L + r] = acc;
}

// coef = Z y (Z column-major n x l, ld ldz): 32 rows x 4 column groups per CTA.
// Batched: instance b = blockIdx.y with n, Z offset, ld and coef offset from tables.
__global__ void __launch_bounds__(128) k_lift(ProjDims d, const double* __restrict__ Z_all, LiftDims ld,
                                              const double* __restrict__ y_all, double* __restrict__ coef_all) {
    __shared__ double red[4][32];
    __shared__ double ys[1024];
    const int b = blockIdx.y;
    const int l = sel_l(d, b);
    const int64_t n = ld.n_arr ? ld.n_arr[b] : ld.n;
    if ((int64_t)blockIdx.x * 32 >= n) return;
    const int64_t ldz = ld.n_arr ? n : ld.ldz;
    const double* Z = Z_all + (ld.zoff ? ld.zoff[b] : 0);
    double* coef = coef_all + (ld.coff ? ld.coff[b] : 0);
    const double* y = y_all + (size_t)b * d.L;
    for (int m = threadIdx.x; m < l; m += 128)
        if (RBF_IN_RANGE(m, 1024)) ys[m] = y[m];  // the projected dimension fits the shared copy
    __syncthreads();
    const int row = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + row;
    double acc = 0.0;
    if (i < n)
        for (int m = grp; m < l; m += 4) acc = fma(Z[(int64_t)m * ldz + i], ys[m], acc);
    red[grp][row] = acc;
    __syncthreads();
    if (grp == 0 && i < n) coef[i] = (red[0][row] + red[1][row]) + (red[2][row] + red[3][row]);
}

}  // namespace

size_t select_ws_bytes(const rbf_ctx* ctx, int l) { return select_ws_bytes_batch(ctx, l, 1); }

rbf_status launch_select_batch(rbf_ctx* ctx, ProjDims d, int method, int rule, double lambda_in, int rank,
                               const double* alpha, const double* beta, const double* Z, LiftDims ld,
                               double* coef, double* curve, void* ws, double* lam_out, int* idx_out,
                               int* rank_out, bool single, const int* rule_arr, const double* lam_arr) {
    const int L = d.L, B = d.B, J = ctx->opt.grid_j;
    const double tlo = ctx->opt.grid_t_lo, thi = ctx->opt.grid_t_hi;
    WsCarve wc(ws);
    double* sigma = wc.take<double>((size_t)L * B);
    double* ftil = wc.take<double>((size_t)(L + 1) * B);
    double* V = wc.take<double>((size_t)L * L * B);
    double* gcv = wc.take<double>((size_t)J * B);
    double* xr = wc.take<double>((size_t)J * B);
    double* ye = wc.take<double>((size_t)J * B);
    double* cvec = wc.take<double>((size_t)L * B);
    double* y = wc.take<double>((size_t)L * B);
    double* work = wc.take<double>((size_t)(L + 2) * B);
    void* svd = (void*)wc.take<char>(svd_ws_bytes_batch(L, B));
    cudaStream_t s = ctx->stream;
    rbf_dev_state* stt = single ? ctx->d_state : nullptr;
    rbf_timer_start(ctx);
    RBF_TRY(launch_projected_svd_batch(ctx, d, alpha, beta, sigma, ftil, V, L, svd, nullptr, nullptr));
    ctx->tim.svd_ms = rbf_timer_stop(ctx);
    rbf_timer_start(ctx);
    if (method == 0) {
        if (rule == RBF_GCV || rule == RBF_LCURVE || rule_arr) {
            k_grid_terms<<<dim3((J + 31) / 32, B), 32, 0, s>>>(d, sigma, ftil, J, tlo, thi, gcv, xr, ye);
            RBF_LAUNCHED(ctx, "k_grid_terms");
        }
        k_choose_lambda<<<B, 1024, 0, s>>>(d, sigma, ftil, J, tlo, thi, rule, lambda_in, rule_arr, lam_arr, gcv, xr,
                                           ye, curve, cvec, lam_out, idx_out, stt);
        RBF_LAUNCHED(ctx, "k_choose_lambda");
    } else {
        k_choose_rank<<<B, 256, 0, s>>>(d, sigma, ftil, rank, curve, cvec, work, rank_out, stt);
        RBF_LAUNCHED(ctx, "k_choose_rank");
    }
    k_vmul<<<dim3((L + 127) / 128, B), 128, 0, s>>>(d, V, L, cvec, y);
    RBF_LAUNCHED(ctx, "k_vmul");
    ctx->tim.select_ms = rbf_timer_stop(ctx);
    rbf_timer_start(ctx);
    const int64_t nmax = ld.nmax;
    if (coef) {
        k_lift<<<dim3((unsigned)((nmax + 31) / 32), B), 128, 0, s>>>(d, Z, ld, y, coef);
        RBF_LAUNCHED(ctx, "k_lift");
    }
    ctx->tim.lift_ms = rbf_timer_stop(ctx);
    return RBF_OK;
}

size_t select_ws_bytes_batch(const rbf_ctx* ctx, int L, int B) {
    const int J = ctx->opt.grid_j;
    size_t b = 0;
    b += ws_align((size_t)L * 8 * B) + ws_align((size_t)(L + 1) * 8 * B) + ws_align((size_t)L * L * 8 * B);
    b += 3 * ws_align((size_t)J * 8 * B);
    b += 3 * ws_align((size_t)(L + 2) * 8 * B);
    return b + svd_ws_bytes_batch(L, B) + 4096;
}

namespace {

void info_from_state(const rbf_dev_state* h, int l, rbf_solve_info* info) {
    info->lambda = h->scal[SC_LAMBDA];
    info->index = h->info[IN_INDEX];
    info->rank = h->info[IN_RANK];
    info->steps = l;
    info->sigma1 = h->scal[SC_SIGMA1];
    info->eta = h->scal[SC_ETA];
    info->rho = h->scal[SC_RHO];
}

rbf_status read_info(rbf_ctx* ctx, rbf_solve_info* info, int l) {
    RBF_CUDA(ctx, cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(rbf_dev_state),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RBF_CUDA(ctx, cudaGetLastError());
    RBF_TRY(rbf_check_all(ctx));
    if (info) info_from_state(ctx->h_state, l, info);
    return RBF_OK;
}

// Enqueue the projected solve of one state (no synchronisation).
rbf_status enqueue_solve(rbf_ctx* ctx, const rbf_gkb_state* st, int method, int rule, double lambda_in, int rank,
                         double* d_coef, double* d_curve) {
    const int l = st->steps_done;
    if (l < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "state has no completed step");
    if (l > 1023) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "projected dimension above 1023");
    RBF_TRY(rbf_ws_reserve(ctx, select_ws_bytes_batch(ctx, l, 1)));
    ProjDims d{1, l, l, nullptr};
    LiftDims ld{nullptr, nullptr, nullptr, st->n, st->ldz, st->n};
    return launch_select_batch(ctx, d, method, rule, lambda_in, rank, st->d_alpha, st->d_beta, st->d_Z, ld, d_coef,
                               d_curve, ctx->ws, nullptr, nullptr, nullptr, true);
}

rbf_status single_solve(rbf_ctx* ctx, const rbf_gkb_state* st, int method, int rule, double lambda_in, int rank,
                        double* d_coef, double* d_curve, rbf_solve_info* info) {
    RBF_TRY(enqueue_solve(ctx, st, method, rule, lambda_in, rank, d_coef, d_curve));
    return read_info(ctx, info, st->steps_done);
}

rbf_status check_rule(rbf_ctx* ctx, int rule, double lambda_in) {
    if (rule != RBF_GCV && rule != RBF_LCURVE && rule != RBF_FIXED && rule != RBF_FIXED_T)
        return rbf_fail(ctx, RBF_ERR_INVALID, "unknown rule %d", rule);
    if (rule == RBF_FIXED && !(lambda_in >= 0.0))
        return rbf_fail(ctx, RBF_ERR_INVALID, "fixed lambda must be >= 0");
    if (rule == RBF_FIXED_T && !(lambda_in >= -300.0 && lambda_in <= 300.0))
        return rbf_fail(ctx, RBF_ERR_INVALID, "fixed t must be finite and within [-300, 300]");
    return RBF_OK;
}

}  // namespace

extern "C" rbf_status rbf_hkt(rbf_ctx* ctx, const rbf_gkb_state* st, int rule, double lambda_in,
                              double* d_coef, double* d_curve, rbf_solve_info* info) {
    RbfRange range_("rbf_hkt");
    if (!ctx) return RBF_ERR_INVALID;
    if (!st || !d_coef) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_hkt: NULL argument");
    return hkt_single(ctx, st, rule, lambda_in, d_coef, info, d_curve);
}

rbf_status hkt_single(rbf_ctx* ctx, const rbf_gkb_state* st, int rule, double lambda_in, double* d_coef,
                      rbf_solve_info* info, double* d_curve) {
    RBF_TRY(check_rule(ctx, rule, lambda_in));
    return single_solve(ctx, st, 0, rule, lambda_in, 0, d_coef, d_curve, info);
}

// HKT for several finished GKB states at once, spread over the context's lanes
// (each lane solves its share one after another; the projected SVD and the
// lambda sweep are single-CTA, latency-bound kernels, so independent solves
// overlap); one synchronisation at the end.
extern "C" rbf_status rbf_hkt_many(rbf_ctx* ctx, int count, const rbf_gkb_state* states, int rule,
                                   double lambda_in, double* const* d_coef, rbf_solve_info* infos, int lanes) {
    RbfRange range_("rbf_hkt_many");
    if (!ctx) return RBF_ERR_INVALID;
    if (count < 1 || !states || !d_coef) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_hkt_many: bad arguments");
    if (lanes < 0 || lanes > rbf_ctx::MAX_LANES)
        return rbf_fail(ctx, RBF_ERR_INVALID, "lanes must be 0 (default) or 1..%d", rbf_ctx::MAX_LANES);
    RBF_TRY(check_rule(ctx, rule, lambda_in));
    for (int i = 0; i < count; ++i)
        if (!d_coef[i]) return rbf_fail(ctx, RBF_ERR_INVALID, "d_coef[%d] is NULL", i);
    int L = lanes == 0 ? rbf_ctx::MAX_LANES : lanes;
    if (L > count) L = count;
    RBF_TRY(rbf_many_slots(ctx, count));
    RBF_TRY(rbf_lanes_fork(ctx, L));
    rbf_status err = RBF_OK;
    for (int i = 0; i < count && err == RBF_OK; ++i) {
        rbf_ctx* c = nullptr;
        err = rbf_lane(ctx, i % L, &c);
        if (err == RBF_OK) err = enqueue_solve(c, &states[i], 0, rule, lambda_in, 0, d_coef[i], nullptr);
        if (err == RBF_OK) {
            cudaError_t e = cudaMemcpyAsync(&ctx->h_many[i], c->d_state, sizeof(rbf_dev_state),
                                            cudaMemcpyDeviceToHost, c->stream);
            if (e != cudaSuccess) err = rbf_fail(c, RBF_ERR_CUDA, "state copy failed: %s", cudaGetErrorString(e));
        }
        if (err != RBF_OK) rbf_fail(ctx, err, "run %d: %s", i, c ? rbf_last_error(c) : "lane");
    }
    rbf_status je = rbf_lanes_join(ctx, L);
    if (err != RBF_OK) return err;
    RBF_TRY(je);
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RBF_CUDA(ctx, cudaGetLastError());
    RBF_TRY(rbf_check_all(ctx));
    if (infos)
        for (int i = 0; i < count; ++i) info_from_state(&ctx->h_many[i], states[i].steps_done, &infos[i]);
    return RBF_OK;
}

extern "C" rbf_status rbf_ine_tsvd(rbf_ctx* ctx, const rbf_gkb_state* st, int rank, double* d_coef,
                                   double* d_curve, rbf_solve_info* info) {
    RbfRange range_("rbf_ine_tsvd");
    if (!ctx) return RBF_ERR_INVALID;
    if (!st || !d_coef) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_ine_tsvd: NULL argument");
    const int l = st->steps_done;
    if (rank < 0 || rank > l) return rbf_fail(ctx, RBF_ERR_INVALID, "rank %d outside [0, l=%d]", rank, l);
    return single_solve(ctx, st, 1, RBF_GCV, 0.0, rank, d_coef, d_curve, info);
}

RBF_CHECK_READER(select)
