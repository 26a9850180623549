// Learned stopping index and lambda on top of HKT (Algorithm 4), and the
// error table that labels its training runs.
//
// rbf_learned_hkt: GKB for feat_steps steps, the 20 stop features, one network
// forward, GKB resumed to the predicted l, the projected Tikhonov solve at the
// predicted t = log10(lambda / s~_1), and an acceptance test: the inputs must
// look like the training set's (standardised features within z_max), t must
// lie in the trained range, and (optionally) the solution norm eta at that t
// must have settled over the last `window` steps.  A rejected prediction falls
// back to the plain rule-driven HKT at l_max.
//
// rbf_hkt_error_table: for several l and a subsampled lambda grid, the max-norm
// error of the reconstructed HKT solution against a reference field at test
// points, from G = Phi(P, X) Z (column i = the reconstruction of z_{i+1}):
// u(l, lambda) = G_l V~ diag(s~ f~ / (s~^2 + lambda^2)) (Sec. 3.3).
#include <cfloat>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

__global__ void k_replicate(const double* __restrict__ alpha, const double* __restrict__ beta, int L,
                            double* __restrict__ a_rep, double* __restrict__ b_rep) {
    const int e = blockIdx.x;
    for (int i = threadIdx.x; i <= L; i += blockDim.x) {
        if (i < L) a_rep[(size_t)e * L + i] = alpha[i];
        b_rep[(size_t)e * (L + 1) + i] = beta[i];
    }
}

constexpr int ET_Q = 8, ET_T = 256;

__global__ void __launch_bounds__(ET_T) k_err_table(const int* __restrict__ ells, int L,
                                                    const double* __restrict__ sigma_all,
                                                    const double* __restrict__ ftil_all,
                                                    const double* __restrict__ V_all, const double* __restrict__ G,
                                                    int64_t ldg, int64_t m, const double* __restrict__ uref, int J,
                                                    double t_lo, double t_hi, int tstride, int Jp,
                                                    double* __restrict__ err) {
    extern __shared__ double sm[];
    __shared__ double red[ET_T / 32][ET_Q + 1];
    const int e = blockIdx.y;
    const int l = ells[e];
    const double* sigma = sigma_all + (size_t)e * L;
    const double* ftil = ftil_all + (size_t)e * (L + 1);
    const double* V = V_all + (size_t)e * L * L;
    const int q0 = blockIdx.x * ET_Q;
    double* cv = sm;
    double* y = sm + ET_Q * L;
    for (int idx = threadIdx.x; idx < ET_Q * l; idx += ET_T) {
        const int q = idx / l, i = idx - q * l;
        double v = 0.0;
        if (q0 + q < Jp) {
            const double lam = sigma[0] * exp10(grid_t((q0 + q) * tstride, J, t_lo, t_hi));
            const double s = sigma[i];
            v = s * ftil[i] / fma(s, s, lam * lam);
        }
        cv[q * L + i] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < ET_Q * l; idx += ET_T) {
        const int q = idx / l, r = idx - q * l;
        double acc = 0.0;
        for (int i = 0; i < l; ++i) acc = fma(V[(int64_t)i * L + r], cv[q * L + i], acc);
        y[q * L + r] = acc;
    }
    __syncthreads();
    double mx[ET_Q];
#pragma unroll
    for (int q = 0; q < ET_Q; ++q) mx[q] = 0.0;
    double umax = 0.0;
    for (int64_t t = threadIdx.x; t < m; t += ET_T) {
        double acc[ET_Q];
#pragma unroll
        for (int q = 0; q < ET_Q; ++q) acc[q] = 0.0;
        for (int r = 0; r < l; ++r) {
            const double g = G[(int64_t)r * ldg + t];
#pragma unroll
            for (int q = 0; q < ET_Q; ++q) acc[q] = fma(g, y[q * L + r], acc[q]);
        }
        const double ur = uref[t];
        umax = fmax(umax, fabs(ur));
#pragma unroll
        for (int q = 0; q < ET_Q; ++q) mx[q] = fmax(mx[q], fabs(acc[q] - ur));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q <= ET_Q; ++q) {
        double v = q < ET_Q ? mx[q] : umax;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(RBF_FULL_MASK, v, o));
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x <= ET_Q) {
        double v = 0.0;
        for (int w = 0; w < ET_T / 32; ++w) v = fmax(v, red[w][threadIdx.x]);
        red[0][threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x < ET_Q && q0 + (int)threadIdx.x < Jp)
        err[(size_t)e * Jp + q0 + threadIdx.x] = red[0][threadIdx.x] / red[0][ET_Q];
}

}  // namespace

extern "C" rbf_status rbf_hkt_error_table(rbf_ctx* ctx, const rbf_gkb_state* st, const double* d_G, int64_t ldg,
                                          int64_t m, const double* d_uref, int n_ell, const int* h_ells,
                                          int t_stride, double* d_err) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!st || !d_G || !d_uref || !h_ells || !d_err || m < 1 || ldg < m || n_ell < 1 || t_stride < 1)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_hkt_error_table: bad argument");
    int L = 0;
    for (int e = 0; e < n_ell; ++e) {
        if (h_ells[e] < 1 || h_ells[e] > st->steps_done)
            return rbf_fail(ctx, RBF_ERR_INVALID, "l = %d outside [1, steps_done = %d]", h_ells[e], st->steps_done);
        L = h_ells[e] > L ? h_ells[e] : L;
    }
    if (L > 1023) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "projected dimension above 1023");
    const int J = ctx->opt.grid_j;
    const int Jp = (J - 1) / t_stride + 1;
    const size_t B = (size_t)n_ell;
    const size_t need = ws_align(B * 4) + ws_align(B * L * 8) + 2 * ws_align(B * (L + 1) * 8) +
                        ws_align(B * L * 8) + ws_align(B * L * L * 8) + svd_ws_bytes_batch(L, n_ell);
    RBF_TRY(rbf_ws_reserve(ctx, need));
    WsCarve wc(ctx->ws);
    int* d_ells = wc.take<int>(B);
    double* a_rep = wc.take<double>(B * L);
    double* b_rep = wc.take<double>(B * (L + 1));
    double* ftil = wc.take<double>(B * (L + 1));
    double* sigma = wc.take<double>(B * L);
    double* V = wc.take<double>(B * L * L);
    void* svd = (void*)wc.take<char>(svd_ws_bytes_batch(L, n_ell));
    RBF_CUDA(ctx, cudaMemcpyAsync(d_ells, h_ells, B * 4, cudaMemcpyHostToDevice, ctx->stream));
    k_replicate<<<n_ell, 256, 0, ctx->stream>>>(st->d_alpha, st->d_beta, L, a_rep, b_rep);
    RBF_LAUNCHED(ctx, "k_replicate");
    ProjDims d{n_ell, L, 0, d_ells};
    RBF_TRY(launch_projected_svd_batch(ctx, d, a_rep, b_rep, sigma, ftil, V, L, svd, nullptr, nullptr));
    const size_t smem = (size_t)2 * ET_Q * L * 8;
    if (smem > 48 * 1024)
        RBF_CUDA(ctx, cudaFuncSetAttribute(k_err_table, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_err_table<<<dim3((unsigned)((Jp + ET_Q - 1) / ET_Q), (unsigned)n_ell), ET_T, smem, ctx->stream>>>(
        d_ells, L, sigma, ftil, V, d_G, ldg, m, d_uref, J, ctx->opt.grid_t_lo, ctx->opt.grid_t_hi, t_stride, Jp,
        d_err);
    RBF_LAUNCHED(ctx, "k_err_table");
    // the host array of l values must outlive the copy
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RBF_OK;
}

extern "C" rbf_status rbf_learned_hkt(rbf_ctx* ctx, const rbf_operator* op, const double* d_f,
                                      const rbf_stopnet* net, rbf_gkb_state* st, double* d_coef,
                                      rbf_learned_info* info) {
    RbfRange range_("rbf_learned_hkt");
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_f || !net || !st || !d_coef || !net->d_params)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_learned_hkt: NULL argument");
    const int j0 = net->feat_steps;
    if (j0 < 1 || j0 > 10 || net->l_min < j0 || net->l_max < net->l_min || net->l_max > st->capacity ||
        net->window < 1 || net->window >= net->l_min || !(net->accept_tol >= 0.0))
        return rbf_fail(ctx, RBF_ERR_INVALID,
                        "rbf_learned_hkt: need 1 <= feat_steps <= 10 <= l_min <= l_max <= capacity, "
                        "1 <= window < l_min, accept_tol >= 0");
    if (net->fallback_rule != RBF_GCV && net->fallback_rule != RBF_LCURVE)
        return rbf_fail(ctx, RBF_ERR_INVALID, "fallback rule must be RBF_GCV or RBF_LCURVE");
    rbf_learned_info out{};
    out.l_pred = 0;
    RBF_TRY(rbf_gkb(ctx, op, d_f, j0, st));
    bool accept = false;
    if (st->steps_done >= j0) {
        float* feat = ctx->d_state->mlp;
        float* yout = ctx->d_state->mlp + 32;
        RBF_TRY(rbf_stop_features(ctx, st, j0, net->d_feat_mean, net->d_feat_std, feat));
        RBF_TRY(rbf_mlp_forward(ctx, net->d_params, feat, 1, yout));
        float hbuf[34];  // features [0, 20), outputs [32, 34)
        RBF_CUDA(ctx, cudaMemcpyAsync(hbuf, feat, sizeof(hbuf), cudaMemcpyDeviceToHost, ctx->stream));
        RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        const double ln_l = (double)hbuf[32] * net->out_std[0] + net->out_mean[0];
        const double t = (double)hbuf[33] * net->out_std[1] + net->out_mean[1];
        bool in_dist = true;
        for (int q = 0; q < RBF_MLP_IN; ++q) {
            if (!std::isfinite(hbuf[q])) in_dist = false;
            if (net->z_max > 0.0 && std::fabs((double)hbuf[q]) > net->z_max) in_dist = false;
        }
        double lp = std::isfinite(ln_l) ? std::exp(std::fmin(ln_l, 30.0)) : (double)net->l_max;
        long lr = std::lround(lp);
        if (lr < net->l_min) lr = net->l_min;
        if (lr > net->l_max) lr = net->l_max;
        out.l_pred = (int)lr;
        out.t_pred = t;
        out.in_distribution = in_dist ? 1 : 0;
        accept = in_dist && std::isfinite(t) && t >= net->t_min && t <= net->t_max;
        if (accept && st->steps_done < out.l_pred && st->breakdown == 0)
            RBF_TRY(rbf_gkb_resume(ctx, op, st, out.l_pred - st->steps_done));
        const int l = st->steps_done;
        const bool eta_test = !std::isinf(net->accept_tol);
        out.eta_change = NAN;
        if (accept && eta_test && l - net->window < 1) accept = false;
        if (accept) {
            rbf_solve_info a{}, b{};
            if (eta_test) {
                rbf_gkb_state prev = *st;
                prev.steps_done = l - net->window;
                RBF_TRY(hkt_single(ctx, &prev, RBF_FIXED_T, t, nullptr, &a));
            }
            RBF_TRY(hkt_single(ctx, st, RBF_FIXED_T, t, d_coef, &b));
            out.solve = b;
            if (eta_test) {
                out.eta_change = b.eta > 0.0 ? std::fabs(b.eta - a.eta) / b.eta : INFINITY;
                accept = out.eta_change <= net->accept_tol;
            }
        }
    }
    out.accepted = accept ? 1 : 0;
    if (!accept) {
        if (st->steps_done < net->l_max && st->breakdown == 0)
            RBF_TRY(rbf_gkb_resume(ctx, op, st, net->l_max - st->steps_done));
        RBF_TRY(hkt_single(ctx, st, net->fallback_rule, 0.0, d_coef, &out.solve));
    }
    out.steps = st->steps_done;
    if (info) *info = out;
    return RBF_OK;
}

// Batched learned stop: all instances run feat_steps steps in one batched GKB,
// their features go through one network forward, and a second batched run
// advances every instance to its own step count (the predicted l when the
// prediction is accepted, l_max otherwise; the first feat_steps steps are
// recomputed there, which keeps each instance's run one uninterrupted GKB).
// The projected solves then use per-instance rules: the predicted t, or the
// fallback rule.
extern "C" rbf_status rbf_batch_learned_hkt(rbf_ctx* ctx, rbf_batch* bt, const rbf_stopnet* net, double* d_coef,
                                            rbf_learned_info* h_info) {
    RbfRange range_("rbf_batch_learned_hkt");
    if (!ctx) return RBF_ERR_INVALID;
    if (!bt || !net || !d_coef || !h_info || !net->d_params || bt->count < 1)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_batch_learned_hkt: NULL argument");
    const int j0 = net->feat_steps;
    if (j0 < 1 || j0 > 10 || net->l_min < j0 || net->l_max < net->l_min || net->l_max > bt->capacity)
        return rbf_fail(ctx, RBF_ERR_INVALID,
                        "rbf_batch_learned_hkt: need 1 <= feat_steps <= 10 <= l_min <= l_max <= capacity");
    if (net->fallback_rule != RBF_GCV && net->fallback_rule != RBF_LCURVE)
        return rbf_fail(ctx, RBF_ERR_INVALID, "fallback rule must be RBF_GCV or RBF_LCURVE");
    const int B = bt->count, L = bt->capacity;
    rbf_batch b1 = *bt;
    b1.steps_limit = nullptr;
    RBF_TRY(rbf_batch_gkb(ctx, &b1, j0, RBF_FORM_C));
    // features of every instance from its first j0 steps
    std::vector<int> larr(B);
    for (int b = 0; b < B; ++b) larr[b] = bt->steps_done[b] < j0 ? bt->steps_done[b] : j0;
    const size_t need = ws_align((size_t)B * 4) + ws_align((size_t)B * L * 8) + ws_align((size_t)B * (L + 1) * 8) +
                        ws_align((size_t)B * L * L * 8) + svd_ws_bytes_batch(L, B) +
                        ws_align((size_t)B * RBF_MLP_IN * 4) + ws_align((size_t)B * RBF_MLP_OUT * 4);
    RBF_TRY(rbf_ws_reserve(ctx, need));
    WsCarve wc(ctx->ws);
    int* d_l = wc.take<int>(B);
    double* sigma = wc.take<double>((size_t)B * L);
    double* ftil = wc.take<double>((size_t)B * (L + 1));
    double* V = wc.take<double>((size_t)B * L * L);
    void* svd = (void*)wc.take<char>(svd_ws_bytes_batch(L, B));
    float* feat = wc.take<float>((size_t)B * RBF_MLP_IN);
    float* yout = wc.take<float>((size_t)B * RBF_MLP_OUT);
    RBF_CUDA(ctx, cudaMemcpyAsync(d_l, larr.data(), sizeof(int) * B, cudaMemcpyHostToDevice, ctx->stream));
    ProjDims d{B, L, 0, d_l};
    RBF_TRY(launch_projected_svd_batch(ctx, d, bt->d_alpha, bt->d_beta, sigma, ftil, V, L, svd, nullptr, nullptr));
    RBF_TRY(launch_stop_features_batch(ctx, bt->d_alpha, bt->d_beta, sigma, L, d_l, B, j0, net->d_feat_mean,
                                       net->d_feat_std, feat));
    RBF_TRY(rbf_mlp_forward(ctx, net->d_params, feat, B, yout));
    std::vector<float> hf((size_t)B * RBF_MLP_IN), hy((size_t)B * RBF_MLP_OUT);
    RBF_CUDA(ctx, cudaMemcpyAsync(hf.data(), feat, hf.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    RBF_CUDA(ctx, cudaMemcpyAsync(hy.data(), yout, hy.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    // per-instance decision
    std::vector<int> limit(B), rules(B);
    std::vector<double> lam_in(B, 0.0), lam_out(B, 0.0);
    int lmax_run = 1;
    for (int b = 0; b < B; ++b) {
        rbf_learned_info out{};
        bool in_dist = larr[b] >= j0;
        for (int q = 0; q < RBF_MLP_IN && in_dist; ++q) {
            const float v = hf[(size_t)b * RBF_MLP_IN + q];
            if (!std::isfinite(v) || (net->z_max > 0.0 && std::fabs((double)v) > net->z_max)) in_dist = false;
        }
        const double ln_l = (double)hy[(size_t)b * 2] * net->out_std[0] + net->out_mean[0];
        const double t = (double)hy[(size_t)b * 2 + 1] * net->out_std[1] + net->out_mean[1];
        const double lp = std::isfinite(ln_l) ? std::exp(std::fmin(ln_l, 30.0)) : (double)net->l_max;
        long lr = std::lround(lp);
        if (lr < net->l_min) lr = net->l_min;
        if (lr > net->l_max) lr = net->l_max;
        const bool accept = in_dist && std::isfinite(t) && t >= net->t_min && t <= net->t_max;
        out.l_pred = larr[b] >= j0 ? (int)lr : 0;
        out.t_pred = t;
        out.in_distribution = in_dist ? 1 : 0;
        out.accepted = accept ? 1 : 0;
        out.eta_change = NAN;
        limit[b] = accept ? (int)lr : net->l_max;
        rules[b] = accept ? RBF_FIXED_T : net->fallback_rule;
        lam_in[b] = accept ? t : 0.0;
        lmax_run = limit[b] > lmax_run ? limit[b] : lmax_run;
        h_info[b] = out;
    }
    rbf_batch b2 = *bt;
    b2.steps_limit = limit.data();
    RBF_TRY(rbf_batch_gkb(ctx, &b2, lmax_run, RBF_FORM_C));
    RBF_TRY(rbf_batch_hkt_each(ctx, bt, rules.data(), lam_in.data(), d_coef, lam_out.data()));
    for (int b = 0; b < B; ++b) {
        h_info[b].steps = bt->steps_done[b];
        h_info[b].solve.lambda = lam_out[b];
        h_info[b].solve.steps = bt->steps_done[b];
        h_info[b].solve.index = -1;
    }
    return RBF_OK;
}
