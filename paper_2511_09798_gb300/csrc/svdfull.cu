// Full SVD of the assembled FP64 collocation matrix (Algorithm 3 step 1) and
// the full-SVD methods on top of it: Tikhonov with GCV (Algorithm 3, eqs.
// gcv_svd and tikh_svd_solution) and TSVD (eq. tsvd_solution).
//
// SVD by one-sided (Hestenes) Jacobi: the columns of W = A are rotated in
// pairs until they are mutually orthogonal (W = U Sigma, V = product of the
// rotations), which keeps the small singular values of these very
// ill-conditioned matrices accurate.  One cooperative kernel per sweep: each
// round pairs the columns by the circle method (n/2 disjoint pairs), one CTA
// per pair: the three dot products |w_i|^2, |w_j|^2, w_i.w_j in one pass, the
// rotation that zeroes w_i.w_j applied to w_i, w_j and v_i, v_j; a bounded
// grid barrier separates the rounds.  Sweeps repeat until no pair needed a
// rotation (|w_i.w_j| <= tol |w_i| |w_j|).  Then sigma_j = |w_j| sorted
// descending, f^ = U^T f = W^T f / sigma, numerical rank r = #{sigma_i >
// N eps sigma_1}, and the solution alpha = V d.
#include <cfloat>
#include <vector>

#include "common.cuh"
#include "grid_sync.cuh"
#include "internal.h"

namespace {

constexpr int JT = 256;
constexpr int JW = JT / 32;
constexpr int MAX_SWEEPS = 40;

// W[j n + i] = A[i lda + j] (column j of A contiguous), V = I.
__global__ void k_fsvd_init(const double* __restrict__ A, int64_t lda, int64_t n, double* __restrict__ W,
                            double* __restrict__ V) {
    __shared__ double t[32][33];
    const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r, j = j0 + threadIdx.x;
        t[r][threadIdx.x] = (i < n && j < n) ? A[i * lda + j] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t j = j0 + r, i = i0 + threadIdx.x;
        if (i < n && j < n) {
            W[j * n + i] = t[threadIdx.x][r];
            V[j * n + i] = i == j ? 1.0 : 0.0;
        }
    }
}

__device__ __forceinline__ int circle_pos(int k, int r, int np) { return k == 0 ? 0 : 1 + (k - 1 + r) % (np - 1); }

// Block-wide sums of three values, result in every thread.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double (*red)[JW]) {
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        red[0][warp] = a;
        red[1][warp] = b;
        red[2][warp] = c;
    }
    __syncthreads();
    a = b = c = 0.0;
#pragma unroll
    for (int w = 0; w < JW; ++w) {
        a += red[0][w];
        b += red[1][w];
        c += red[2][w];
    }
}

__global__ void __launch_bounds__(JT) k_jacobi_sweep(double* __restrict__ W, double* __restrict__ V, int64_t n,
                                                     int np, double tol, rbf_dev_state* __restrict__ stt,
                                                     unsigned* __restrict__ bar, int group, long long budget,
                                                     int* __restrict__ rot_out) {
    __shared__ double red[3][JW];
    int nrot = 0;
    for (int r = 0; r < np - 1; ++r) {
        for (int p = blockIdx.x; p < np / 2; p += gridDim.x) {
            int i = circle_pos(p, r, np), j = circle_pos(np - 1 - p, r, np);
            if (i >= n || j >= n) continue;  // the dummy column of an odd n
            if (i > j) {
                const int t = i;
                i = j;
                j = t;
            }
            double* wi = W + (int64_t)i * n;
            double* wj = W + (int64_t)j * n;
            double a = 0.0, b = 0.0, g = 0.0;
            for (int64_t k = threadIdx.x; k < n; k += JT) {
                const double x = wi[k], y = wj[k];
                a = fma(x, x, a);
                b = fma(y, y, b);
                g = fma(x, y, g);
            }
            block_sum3(a, b, g, red);
            if (g == 0.0 || !(fabs(g) > tol * sqrt(a) * sqrt(b))) continue;
            const double zeta = (b - a) / (2.0 * g);
            const double t = fabs(zeta) > 1e150 ? 0.5 / zeta
                                                 : copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
            const double c = 1.0 / sqrt(fma(t, t, 1.0));
            const double s = c * t;
            for (int64_t k = threadIdx.x; k < n; k += JT) {
                const double x = wi[k], y = wj[k];
                wi[k] = c * x - s * y;
                wj[k] = fma(s, x, c * y);
            }
            double* vi = V + (int64_t)i * n;
            double* vj = V + (int64_t)j * n;
            for (int64_t k = threadIdx.x; k < n; k += JT) {
                const double x = vi[k], y = vj[k];
                vi[k] = c * x - s * y;
                vj[k] = fma(s, x, c * y);
            }
            ++nrot;
        }
        if (!grid_sync(stt, bar, group, budget)) return;
    }
    if (threadIdx.x == 0) rot_out[blockIdx.x] = nrot;
}

// sigma_j = |w_j| (one CTA per column)
__global__ void __launch_bounds__(JT) k_colnorm(const double* __restrict__ W, int64_t n, double* __restrict__ sig) {
    __shared__ double red[3][JW];
    const double* w = W + (int64_t)blockIdx.x * n;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += JT) a = fma(w[k], w[k], a);
    block_sum3(a, b, c, red);
    if (threadIdx.x == 0) sig[blockIdx.x] = sqrt(a);
}

// perm[rank] = j, descending sigma, ties by index
__global__ void k_sort_rank(const double* __restrict__ sig, int64_t n, int* __restrict__ perm,
                            double* __restrict__ sig_sorted) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double s = sig[j];
    int64_t rank = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double t = sig[i];
        rank += (t > s || (t == s && i < j)) ? 1 : 0;
    }
    perm[rank] = (int)j;
    sig_sorted[rank] = s;
}

// fhat[k] = w_{perm k} . f / sigma_k (0 for a zero column)
__global__ void __launch_bounds__(JT) k_fhat(const double* __restrict__ W, int64_t n, const int* __restrict__ perm,
                                             const double* __restrict__ sig_sorted, const double* __restrict__ f,
                                             double* __restrict__ fhat) {
    __shared__ double red[3][JW];
    const int kk = blockIdx.x;
    const double* w = W + (int64_t)perm[kk] * n;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += JT) a = fma(w[k], f[k], a);
    block_sum3(a, b, c, red);
    if (threadIdx.x == 0) fhat[kk] = sig_sorted[kk] > 0.0 ? a / sig_sorted[kk] : 0.0;
}

// rank r and s_perp = sum_{i >= r} fhat_i^2 (one thread; O(n))
__global__ void k_fsvd_rank(const double* __restrict__ sig, const double* __restrict__ fhat, int64_t n,
                            int* __restrict__ r_out, double* __restrict__ sperp_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double thr = (double)n * DBL_EPSILON * sig[0];
    int64_t r = 0;
    while (r < n && sig[r] > thr && sig[0] > 0.0) ++r;
    double sp = 0.0;
    for (int64_t i = r; i < n; ++i) sp = fma(fhat[i], fhat[i], sp);
    *r_out = (int)r;
    *sperp_out = sp;
}

// Tikhonov GCV on the grid: (sum_{i<r} (1-phi_i)^2 fhat_i^2 + s_perp) / ((n - r) + sum_{i<r} (1-phi_i))^2
__global__ void k_fsvd_gcv(const double* __restrict__ sig, const double* __restrict__ fhat, int64_t n,
                           const int* __restrict__ r_in, const double* __restrict__ sperp, int J, double t_lo,
                           double t_hi, double* __restrict__ gcv) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= J) return;
    const int r = *r_in;
    const double lam = sig[0] * exp10(grid_t(t, J, t_lo, t_hi));
    const double l2 = lam * lam;
    double num = 0.0, den = (double)(n - r);
    for (int i = 0; i < r; ++i) {
        const double s = sig[i];
        const double q = l2 / fma(s, s, l2);
        num = fma(q * q, fhat[i] * fhat[i], num);
        den += q;
    }
    gcv[t] = (num + *sperp) / (den * den);
}

// TSVD GCV over k = 1..min(r, n-1): (sum_{k<=i<r} fhat_i^2 + s_perp) / (n - k)^2
__global__ void k_fsvd_gcv_rank(const double* __restrict__ fhat, int64_t n, const int* __restrict__ r_in,
                                const double* __restrict__ sperp, double* __restrict__ curve) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int r = *r_in;
    const int64_t kmax = r < n - 1 ? r : n - 1;
    if (k > kmax) return;
    double s = *sperp;
    for (int64_t i = r - 1; i >= k; --i) s = fma(fhat[i], fhat[i], s);
    const double d = (double)(n - k);
    curve[k - 1] = s / (d * d);
}

// argmin with lowest index on ties (one block); method 0: Tikhonov (index into
// the grid), 1: TSVD (k = index + 1).  Writes d_i and the choice.
__global__ void k_fsvd_choose(const double* __restrict__ curve, int count, int method, int fixed_mode,
                              double lambda_in, int rank_in, const double* __restrict__ sig,
                              const double* __restrict__ fhat, const int* __restrict__ r_in, int J, double t_lo,
                              double t_hi, double* __restrict__ d, int64_t n, rbf_dev_state* __restrict__ stt) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    __shared__ double lam_s;
    __shared__ int k_s;
    double best = INFINITY;
    int besti = 0x7fffffff;
    if (!fixed_mode)
        for (int t = threadIdx.x; t < count; t += blockDim.x) {
            double v = curve[t];
            if (isnan(v)) v = INFINITY;
            if (v < best || (v == best && t < besti)) { best = v; besti = t; }
        }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            const double ov = bv[threadIdx.x + off], mv = bv[threadIdx.x];
            const int oi = bi[threadIdx.x + off], mi = bi[threadIdx.x];
            if (ov < mv || (ov == mv && oi < mi)) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int r = *r_in;
    if (threadIdx.x == 0) {
        int idx = bi[0];
        if (idx < 0 || idx >= count) idx = 0;
        if (method == 0) {
            lam_s = fixed_mode ? lambda_in : sig[0] * exp10(grid_t(idx, J, t_lo, t_hi));
            k_s = r;
            stt->info[IN_INDEX] = fixed_mode ? -1 : idx;
            stt->scal[SC_LAMBDA] = lam_s;
        } else {
            k_s = fixed_mode ? rank_in : idx + 1;
            lam_s = 0.0;
            stt->info[IN_RANK] = k_s;
            stt->scal[SC_LAMBDA] = 0.0;
        }
        stt->scal[SC_SIGMA1] = sig[0];
    }
    __syncthreads();
    const double l2 = lam_s * lam_s;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double v = 0.0;
        if (method == 0) {
            if (i < r) v = sig[i] * fhat[i] / fma(sig[i], sig[i], l2);
        } else if (i < k_s && sig[i] > 0.0) {
            v = fhat[i] / sig[i];
        }
        d[i] = v;
    }
}

// coef[row] = sum_k V[perm k][row] d_k (V column-major; one thread per row)
__global__ void k_fsvd_lift(const double* __restrict__ V, int64_t n, const int* __restrict__ perm,
                            const double* __restrict__ d, double* __restrict__ coef) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    double acc = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double dk = d[k];
        if (dk != 0.0) acc = fma(V[(int64_t)perm[k] * n + row], dk, acc);
    }
    coef[row] = acc;
}

// out[:, k] = V[:, perm k] (column-major)
__global__ void k_gather_cols(const double* __restrict__ V, int64_t n, const int* __restrict__ perm,
                              double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k = blockIdx.y;
    if (i < n) out[k * n + i] = V[(int64_t)perm[k] * n + i];
}

struct FsvdWs {
    double *W, *V, *sig, *sig_sorted, *fhat, *curve, *d, *sperp;
    int *perm, *r, *rot;
    unsigned* bar;
};

size_t fsvd_ws_bytes(int64_t n, int G, int bar_k, int J) {
    return 2 * ws_align((size_t)n * n * 8) + 5 * ws_align((size_t)n * 8) + ws_align((size_t)(J > n ? J : n) * 8) +
           ws_align(8) + ws_align((size_t)n * 4) + ws_align(4) + ws_align((size_t)G * 4) +
           ws_align((size_t)(bar_k + 2) * BAR_STRIDE * 4) + 4096;
}

// The SVD itself: W, V, sig_sorted, perm, fhat (when f given), r, s_perp.
rbf_status fsvd_run(rbf_ctx* ctx, const rbf_operator* op, const double* f, FsvdWs* out, int* sweeps_out) {
    const int64_t n = op->n;
    if (op->storage != RBF_ASSEMBLED || op->precision != RBF_FP64 || !op->d_A)
        return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "the full SVD needs an assembled FP64 operator");
    if (n < 2 || n > 8192) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "full SVD for 2 <= n <= 8192 (n = %lld)",
                                           (long long)n);
    int occ = 0;
    RBF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_jacobi_sweep, JT, 0));
    const int np = (int)(n + (n & 1));
    int G = ctx->sm_count * (occ < 1 ? 1 : occ);
    if (G > np / 2) G = np / 2;
    int group = 1;
    while (group * group < G) ++group;
    const int bar_k = (G + group - 1) / group;
    const int J = ctx->opt.grid_j;
    RBF_TRY(rbf_ws_reserve(ctx, fsvd_ws_bytes(n, G, bar_k, J)));
    WsCarve wc(ctx->ws);
    FsvdWs w;
    w.W = wc.take<double>((size_t)n * n);
    w.V = wc.take<double>((size_t)n * n);
    w.sig = wc.take<double>((size_t)n);
    w.sig_sorted = wc.take<double>((size_t)n);
    w.fhat = wc.take<double>((size_t)n);
    w.d = wc.take<double>((size_t)n);
    w.curve = wc.take<double>((size_t)(J > n ? J : n));
    w.sperp = wc.take<double>(1);
    w.perm = wc.take<int>((size_t)n);
    w.r = wc.take<int>(1);
    w.rot = wc.take<int>((size_t)G);
    w.bar = wc.take<unsigned>((size_t)(bar_k + 2) * BAR_STRIDE);
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaMemsetAsync(w.bar, 0, (size_t)(bar_k + 2) * BAR_STRIDE * sizeof(unsigned), s));
    RBF_CUDA(ctx, cudaMemsetAsync(&ctx->d_state->info[IN_ERR], 0, sizeof(int), s));
    RBF_CUDA(ctx, cudaMemsetAsync(&ctx->d_state->info[IN_DONE], 0, sizeof(int), s));
    dim3 tb(32, 8), tg((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    k_fsvd_init<<<tg, tb, 0, s>>>((const double*)op->d_A, op->lda, n, w.W, w.V);
    RBF_LAUNCHED(ctx, "k_fsvd_init");
    const double tol = 8.0 * DBL_EPSILON;
    long long budget = 1LL << 23;
    std::vector<int> rot((size_t)G);
    int sweeps = 0;
    for (; sweeps < MAX_SWEEPS; ++sweeps) {
        double* Wp = w.W;
        double* Vp = w.V;
        int64_t nn = n;
        int npp = np;
        double tl = tol;
        rbf_dev_state* stt = ctx->d_state;
        unsigned* bar = w.bar;
        int grp = group;
        int* rp = w.rot;
        void* args[] = {&Wp, &Vp, &nn, &npp, &tl, &stt, &bar, &grp, &budget, &rp};
        RBF_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_jacobi_sweep, dim3(G), dim3(JT), args, 0, s));
        ctx->launches++;
        int err = 0;
        RBF_CUDA(ctx, cudaMemcpyAsync(rot.data(), w.rot, sizeof(int) * G, cudaMemcpyDeviceToHost, s));
        RBF_CUDA(ctx, cudaMemcpyAsync(&err, &ctx->d_state->info[IN_ERR], sizeof(int), cudaMemcpyDeviceToHost, s));
        RBF_CUDA(ctx, cudaStreamSynchronize(s));
        if (err) return rbf_fail(ctx, (rbf_status)err, "a bounded grid barrier of the Jacobi sweep gave up");
        long long total = 0;
        for (int q = 0; q < G; ++q) total += rot[q];
        if (total == 0) {
            ++sweeps;
            break;
        }
    }
    k_colnorm<<<(unsigned)n, JT, 0, s>>>(w.W, n, w.sig);
    RBF_LAUNCHED(ctx, "k_colnorm");
    k_sort_rank<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.sig, n, w.perm, w.sig_sorted);
    RBF_LAUNCHED(ctx, "k_sort_rank");
    if (f) {
        k_fhat<<<(unsigned)n, JT, 0, s>>>(w.W, n, w.perm, w.sig_sorted, f, w.fhat);
        RBF_LAUNCHED(ctx, "k_fhat");
        k_fsvd_rank<<<1, 32, 0, s>>>(w.sig_sorted, w.fhat, n, w.r, w.sperp);
        RBF_LAUNCHED(ctx, "k_fsvd_rank");
    }
    *out = w;
    if (sweeps_out) *sweeps_out = sweeps;
    return RBF_OK;
}

rbf_status read_state(rbf_ctx* ctx) {
    RBF_CUDA(ctx, cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(rbf_dev_state), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RBF_CUDA(ctx, cudaGetLastError());
    return RBF_OK;
}

}  // namespace

extern "C" rbf_status rbf_svd_full(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, double* d_sigma,
                                   double* d_fhat, double* d_V, int* sweeps) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_sigma || (d_fhat && !d_f)) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_svd_full: bad argument");
    FsvdWs w;
    RBF_TRY(fsvd_run(ctx, op, d_fhat ? d_f : nullptr, &w, sweeps));
    const int64_t n = op->n;
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaMemcpyAsync(d_sigma, w.sig_sorted, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (d_fhat) RBF_CUDA(ctx, cudaMemcpyAsync(d_fhat, w.fhat, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (d_V) {
        k_gather_cols<<<dim3((unsigned)((n + 255) / 256), (unsigned)n), 256, 0, s>>>(w.V, n, w.perm, d_V);
        RBF_LAUNCHED(ctx, "k_gather_cols");
    }
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    return RBF_OK;
}

extern "C" rbf_status rbf_tikhonov(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int rule,
                                   double lambda_in, double* d_coef, rbf_solve_info* info) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_f || !d_coef) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_tikhonov: NULL argument");
    if (rule != RBF_GCV && rule != RBF_FIXED) return rbf_fail(ctx, RBF_ERR_INVALID, "rule must be RBF_GCV or RBF_FIXED");
    if (rule == RBF_FIXED && !(lambda_in >= 0.0)) return rbf_fail(ctx, RBF_ERR_INVALID, "fixed lambda must be >= 0");
    FsvdWs w;
    int sweeps = 0;
    RBF_TRY(fsvd_run(ctx, op, d_f, &w, &sweeps));
    const int64_t n = op->n;
    const int J = ctx->opt.grid_j;
    cudaStream_t s = ctx->stream;
    const double tlo = ctx->opt.grid_t_lo, thi = ctx->opt.grid_t_hi;
    if (rule == RBF_GCV) {
        k_fsvd_gcv<<<(J + 127) / 128, 128, 0, s>>>(w.sig_sorted, w.fhat, n, w.r, w.sperp, J, tlo, thi, w.curve);
        RBF_LAUNCHED(ctx, "k_fsvd_gcv");
    }
    k_fsvd_choose<<<1, 1024, 0, s>>>(w.curve, J, 0, rule == RBF_FIXED, lambda_in, 0, w.sig_sorted, w.fhat, w.r, J,
                                      tlo, thi, w.d, n, ctx->d_state);
    RBF_LAUNCHED(ctx, "k_fsvd_choose");
    k_fsvd_lift<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(w.V, n, w.perm, w.d, d_coef);
    RBF_LAUNCHED(ctx, "k_fsvd_lift");
    int r = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&r, w.r, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_TRY(read_state(ctx));
    if (info) {
        info->lambda = ctx->h_state->scal[SC_LAMBDA];
        info->index = ctx->h_state->info[IN_INDEX];
        info->rank = r;
        info->steps = sweeps;
        info->sigma1 = ctx->h_state->scal[SC_SIGMA1];
        info->eta = 0.0;
        info->rho = 0.0;
    }
    return RBF_OK;
}

extern "C" rbf_status rbf_tsvd(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int rank, double* d_coef,
                               rbf_solve_info* info) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_f || !d_coef) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_tsvd: NULL argument");
    if (rank < 0 || rank > op->n) return rbf_fail(ctx, RBF_ERR_INVALID, "rank %d outside [0, n]", rank);
    FsvdWs w;
    int sweeps = 0;
    RBF_TRY(fsvd_run(ctx, op, d_f, &w, &sweeps));
    const int64_t n = op->n;
    cudaStream_t s = ctx->stream;
    if (rank == 0) {
        k_fsvd_gcv_rank<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(w.fhat, n, w.r, w.sperp, w.curve);
        RBF_LAUNCHED(ctx, "k_fsvd_gcv_rank");
    }
    int r = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&r, w.r, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    const int kmax = (int)(r < n - 1 ? r : n - 1);
    if (rank == 0 && kmax < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "numerical rank 0: no TSVD solution");
    k_fsvd_choose<<<1, 1024, 0, s>>>(w.curve, kmax, 1, rank != 0, 0.0, rank, w.sig_sorted, w.fhat, w.r,
                                      ctx->opt.grid_j, ctx->opt.grid_t_lo, ctx->opt.grid_t_hi, w.d, n, ctx->d_state);
    RBF_LAUNCHED(ctx, "k_fsvd_choose");
    k_fsvd_lift<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(w.V, n, w.perm, w.d, d_coef);
    RBF_LAUNCHED(ctx, "k_fsvd_lift");
    RBF_TRY(read_state(ctx));
    if (info) {
        info->lambda = 0.0;
        info->index = -1;
        info->rank = ctx->h_state->info[IN_RANK];
        info->steps = sweeps;
        info->sigma1 = ctx->h_state->scal[SC_SIGMA1];
        info->eta = 0.0;
        info->rho = 0.0;
    }
    return RBF_OK;
}
