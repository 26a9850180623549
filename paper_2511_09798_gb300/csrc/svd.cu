// Projected SVD of the lower-bidiagonal C_l ((l+1) x l) of Algorithms 2 and 4:
// C_l = U~ S~ V~^T, f~ = U~^T (beta_1 e_1).
//
// On GB300 a dependent FP64 operation costs ~64 cycles (FP64 division ~640), so
// a sequential bidiagonal QR sweep would take tens of milliseconds.  This
// implementation instead works on the Golub-Kahan tridiagonal T (order 2l+1,
// zero diagonal, off-diagonal alpha_1, beta_2, alpha_2, ..., alpha_l, beta_{l+1},
// eigenvalues +-s~_i and 0, eigenvectors (u~_i, v~_i interleaved)/sqrt(2)),
// which exposes parallelism over the singular values:
//
//  1. k_tgk_bisect  one warp per singular value: 32-point multisection on the
//     IEEE bit pattern of the shift (uniform steps in the bit pattern of a
//     positive double are nearly geometric), Sturm counts from the
//     division-free three-term recurrence of the leading principal minors with
//     power-of-two rescaling.  Converges to adjacent doubles in <= 14 rounds.
//  2. k_tgk_vectors one thread per singular value: twisted factorization
//     (top-down and bottom-up LDL^T of T - s I, twist where |gamma| is
//     smallest) gives the eigenvector without iteration.
//  3. k_tgk_clusters one warp per cluster of close singular values (relative
//     gap < cluster_tol; as many CTAs as needed for one cluster per warp):
//     three steps of inverse iteration with the stored
//     factorizations, all members in parallel lanes, Gram-Schmidt in order
//     (the scheme of LAPACK's dstein), so the cluster basis is orthonormal.
//  4. k_tgk_finalize split into u~ and v~, normalise, f~_i = beta_1 u~_i[0];
//     f~_{l+1} = beta_1 / |u| with u the null vector of C^T (u_1 = 1,
//     u_{j+1} = -alpha_j u_j / beta_{j+1}), accumulated in log space.
// Everything is FP64.
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int BS_WARPS = 4;
constexpr int SVD_MAX_L = 8192;  // bidiagonal dimension (shared memory: 2 L doubles)

__device__ __forceinline__ int proj_l(const ProjDims& d, int b) { return d.l_arr ? d.l_arr[b] : d.l; }

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double bitsd(long long b) { return __longlong_as_double(b); }

// Normalised off-diagonal of T: e_{2m} = alpha_{m+1}, e_{2m+1} = beta_{m+2}; / bound.
__device__ void load_e(const double* __restrict__ alpha, const double* __restrict__ beta, int l,
                       double* e, double* bound_out) {
    __shared__ double red[32];
    const int ne = 2 * l;
    for (int k = threadIdx.x; k < ne; k += blockDim.x) e[k] = (k & 1) ? beta[(k >> 1) + 1] : alpha[k >> 1];
    __syncthreads();
    double b = 0.0;
    for (int k = threadIdx.x; k < ne; k += blockDim.x) {
        double g = fabs(e[k]) + (k + 1 < ne ? fabs(e[k + 1]) : 0.0);
        b = fmax(b, g);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = fmax(b, __shfl_xor_sync(RBF_FULL_MASK, b, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
        red[0] = t > 0.0 ? t : 1.0;
    }
    __syncthreads();
    const double bound = red[0];
    const double inv = 1.0 / bound;
    for (int k = threadIdx.x; k < ne; k += blockDim.x) e[k] *= inv;
    __syncthreads();
    *bound_out = bound;
}

// power of two that brings max(|a|, |b|) near 1 (integer ops on the exponents)
__device__ __forceinline__ double rescale_factor(double a, double b) {
    int ea = (__double2hiint(a) >> 20) & 0x7ff;
    int eb = (__double2hiint(b) >> 20) & 0x7ff;
    int e = max(ea, eb);                 // biased exponent of the larger
    int t = 2046 - e;                    // biased exponent of 2^-(e - 1023)
    t = max(1, min(2046, t));
    return __hiloint2double(t << 20, 0);
}

// number of eigenvalues of the normalised T below x > 0
__device__ int sturm_count(const double* __restrict__ e2, int nt, double x) {
    double pm2 = 1.0, pm1 = -x;
    int neg = 1;  // d_0 = -x < 0
    for (int k = 1; k < nt; ++k) {
        double p = fma(-x, pm1, -e2[k - 1] * pm2);
        if ((dbits(p) << 1) == 0) p = -1e-300 * pm1;  // zero pivot counts as negative
        neg += (int)(sign_bit(p) ^ sign_bit(pm1));
        pm2 = pm1;
        pm1 = p;
        if ((k & 7) == 0) {
            double f = rescale_factor(pm1, pm2);
            pm1 *= f;
            pm2 *= f;
        }
    }
    return neg;
}

__global__ void k_tgk_bisect(ProjDims d, const double* __restrict__ alpha_all,
                             const double* __restrict__ beta_all, double* __restrict__ sigma_all,
                             double* __restrict__ bound_all) {
    extern __shared__ double sh[];
    const int b = blockIdx.y;
    const int l = proj_l(d, b);
    if (l < 1) return;
    const double* alpha = alpha_all + (size_t)b * d.L;
    const double* beta = beta_all + (size_t)b * (d.L + 1);
    double* sigma = sigma_all + (size_t)b * d.L;
    double* e2 = sh;  // 2l: the normalised off-diagonal, squared in place
    double bound;
    load_e(alpha, beta, l, e2, &bound);
    for (int k = threadIdx.x; k < 2 * l; k += blockDim.x) e2[k] = e2[k] * e2[k];
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) bound_all[b] = bound;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * BS_WARPS + warp;  // descending index
    if (i >= l) return;
    const int m = l - 1 - i;                     // ascending rank
    const int nt = 2 * l + 1;
    long long lo = 0, hi = dbits(1.0 + 1.0 / 1024.0);
    for (int round = 0; round < 24 && hi - lo > 1; ++round) {
        const long long dd = hi - lo;
        long long xb;
        if (dd >= 33) xb = lo + (dd / 33) * (lane + 1);
        else xb = lo + min((long long)(lane + 1), dd - 1);
        const int cnt = sturm_count(e2, nt, bitsd(xb)) - (l + 1);
        const unsigned above = __ballot_sync(RBF_FULL_MASK, cnt > m);
        const long long x_prev = __shfl_up_sync(RBF_FULL_MASK, xb, 1);
        if (above == 0) {
            lo = __shfl_sync(RBF_FULL_MASK, xb, 31);
        } else {
            const int f = __ffs(above) - 1;
            const long long nh = __shfl_sync(RBF_FULL_MASK, xb, f);
            const long long nl = __shfl_sync(RBF_FULL_MASK, x_prev, f);
            if (f > 0) lo = nl;
            hi = nh;
        }
    }
    if (lane == 0) sigma[i] = 0.5 * (bitsd(lo) + bitsd(hi)) * bound;
}

// Twisted factorization eigenvector of the normalised T for s = sigma_i / bound.
// Scratch per instance (k-major, stride L): invdp[k][i] = 1/d+_k,
// rp[k][i] = e_k / d+_k, rm[k][i] = e_{k-1} / d-_k.  Output X[i * NT + k].
__global__ void k_tgk_vectors(ProjDims d, const double* __restrict__ alpha_all,
                              const double* __restrict__ beta_all, const double* __restrict__ sigma_all,
                              const double* __restrict__ bound_all, double* __restrict__ invdp_all,
                              double* __restrict__ rp_all, double* __restrict__ rm_all,
                              double* __restrict__ X_all) {
    extern __shared__ double e[];
    const int b = blockIdx.y;
    const int l = proj_l(d, b);
    if (l < 1) return;
    const int L = d.L, NT = 2 * d.L + 1;
    const size_t sc = (size_t)b * NT * L;
    double* invdp = invdp_all + sc;
    double* rp = rp_all + sc;
    double* rm = rm_all + sc;
    double* X = X_all + sc;
    double bound;
    load_e(alpha_all + (size_t)b * L, beta_all + (size_t)b * (L + 1), l, e, &bound);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= l) return;
    const int nt = 2 * l + 1;
    const double s = sigma_all[(size_t)b * L + i] / bound;
    const double pivmin = -DBL_MIN;
    // top-down: d+_0 = -s, d+_k = -s - e_{k-1} rp_{k-1}
    double dd = -s;
    for (int k = 0; k < nt; ++k) {
        if (k > 0) dd = fma(-e[k - 1], rp[(size_t)(k - 1) * L + i], -s);
        if (dd == 0.0) dd = pivmin;
        const double inv = 1.0 / dd;
        invdp[(size_t)k * L + i] = inv;
        if (k < nt - 1) rp[(size_t)k * L + i] = e[k] * inv;
        X[(size_t)i * NT + k] = dd;  // keep d+ for gamma
    }
    // bottom-up: d-_{nt-1} = -s, d-_k = -s - e_k rm_{k+1}; gamma_k = d+_k + d-_k + s
    double dm = -s;
    double best = 1e308;
    int r = nt - 1;
    for (int k = nt - 1; k >= 0; --k) {
        if (k < nt - 1) dm = fma(-e[k], rm[(size_t)(k + 1) * L + i], -s);
        if (dm == 0.0) dm = pivmin;
        if (k > 0) rm[(size_t)k * L + i] = e[k - 1] / dm;
        const double gm = fabs(X[(size_t)i * NT + k] + dm + s);
        if (gm < best) {
            best = gm;
            r = k;
        }
    }
    // x_r = 1; upward x_k = -rp_k x_{k+1}; downward x_k = -rm_k x_{k-1}
    double* x = X + (size_t)i * NT;
    x[r] = 1.0;
    double nrm2 = 1.0;
    for (int k = r - 1; k >= 0; --k) {
        x[k] = -rp[(size_t)k * L + i] * x[k + 1];
        nrm2 = fma(x[k], x[k], nrm2);
    }
    for (int k = r + 1; k < nt; ++k) {
        x[k] = -rm[(size_t)k * L + i] * x[k - 1];
        nrm2 = fma(x[k], x[k], nrm2);
    }
    const double inv = rsqrt(nrm2);
    for (int k = 0; k < nt; ++k) x[k] *= inv;
}

// Clusters of close singular values: inverse iteration (3 steps) with the
// stored LDL^T factors of T - s_a I, all members in parallel lanes, then
// modified Gram-Schmidt in order.  One block per instance, one warp per cluster.
constexpr int CL_WARPS = 8;
constexpr int CL_MAX = 32;

// Grid (B, gy): CTA y takes the clusters of index y CL_WARPS .. y CL_WARPS +
// CL_WARPS - 1 (in the order of the descending singular values), one per warp;
// every CTA finds them with the same scan.  A cluster's member vectors are
// iterated in place in X.
__global__ void k_tgk_clusters(ProjDims d, const double* __restrict__ sigma_all, double tol,
                               const double* __restrict__ invdp_all, const double* __restrict__ rp_all,
                               double* __restrict__ X_all) {
    __shared__ int own_start[CL_WARPS], own_end[CL_WARPS];
    const int b = blockIdx.x;
    const int l = proj_l(d, b);
    if (l < 1) return;
    const int L = d.L, NT = 2 * d.L + 1;
    const size_t sc = (size_t)b * NT * L;
    const double* sigma = sigma_all + (size_t)b * L;
    const double* invdp = invdp_all + sc;
    const double* rp = rp_all + sc;
    double* X = X_all + sc;
    if (threadIdx.x < CL_WARPS) own_start[threadIdx.x] = -1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int c0 = blockIdx.y * CL_WARPS;
        int c = 0;
        int i = 0;
        while (i < l && c < c0 + CL_WARPS) {
            int j = i;
            while (j + 1 < l && j - i + 1 < CL_MAX && fabs(sigma[j] - sigma[j + 1]) < tol * sigma[j]) ++j;
            if (j > i) {
                if (c >= c0) {
                    own_start[c - c0] = i;
                    own_end[c - c0] = j;
                }
                ++c;
            }
            i = j + 1;
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = 2 * l + 1;
    const int a0 = own_start[warp];
    if (a0 < 0) return;
    const int a1 = own_end[warp];
    const int mcnt = a1 - a0 + 1;
    double* y = X + (size_t)a0 * NT;  // member vectors of this warp's cluster, in place
    // deterministic start vectors
    for (int a = 0; a < mcnt; ++a)
        for (int k = lane; k < nt; k += 32) y[(size_t)a * NT + k] = sin(0.7 * (double)(k + 1) * (a + 1) + 0.3);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
        // lane a solves (T - s_a I) x = y_a:  L D L^T with L_{k+1,k} = rp_k
        if (lane < mcnt) {
            const int ia = a0 + lane;
            double* v = y + (size_t)lane * NT;
            for (int k = 1; k < nt; ++k) v[k] = fma(-rp[(size_t)(k - 1) * L + ia], v[k - 1], v[k]);
            for (int k = 0; k < nt; ++k) v[k] *= invdp[(size_t)k * L + ia];
            for (int k = nt - 2; k >= 0; --k) v[k] = fma(-rp[(size_t)k * L + ia], v[k + 1], v[k]);
        }
        __syncwarp();
        // modified Gram-Schmidt in member order
        for (int a = 0; a < mcnt; ++a) {
            double* va = y + (size_t)a * NT;
            for (int bb = 0; bb < a; ++bb) {
                const double* vb = y + (size_t)bb * NT;
                double dot = 0.0;
                for (int k = lane; k < nt; k += 32) dot = fma(vb[k], va[k], dot);
                dot = warp_sum(dot);
                for (int k = lane; k < nt; k += 32) va[k] = fma(-dot, vb[k], va[k]);
                __syncwarp();
            }
            double n2 = 0.0;
            for (int k = lane; k < nt; k += 32) n2 = fma(va[k], va[k], n2);
            n2 = warp_sum(n2);
            const double inv = rsqrt(n2);
            for (int k = lane; k < nt; k += 32) va[k] *= inv;
            __syncwarp();
        }
    }
}

// Split the eigenvectors into u~, v~ (normalised), write V~ (and U~ when
// asked: column i = u~_i, l+1 entries, ld ldu) and f~.  One block per instance.
__global__ void k_tgk_finalize(ProjDims d, const double* __restrict__ alpha_all,
                               const double* __restrict__ beta_all, const double* __restrict__ X_all,
                               double* __restrict__ ftil_all, double* __restrict__ V_all, int64_t ldv,
                               rbf_dev_state* __restrict__ stt, const double* __restrict__ sigma_all,
                               double* __restrict__ sigma1_out, double* __restrict__ ftil_last_out,
                               double* __restrict__ U_all, int64_t ldu) {
    extern __shared__ double Ls[];  // l + 1
    __shared__ double red[32];
    const int b = blockIdx.x;
    const int l = proj_l(d, b);
    if (l < 1) return;
    const int L = d.L, NT = 2 * d.L + 1;
    const double* alpha = alpha_all + (size_t)b * L;
    const double* beta = beta_all + (size_t)b * (L + 1);
    const double* X = X_all + (size_t)b * NT * L;
    double* ftil = ftil_all + (size_t)b * (L + 1);
    double* V = V_all + (size_t)b * L * ldv;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nt = 2 * l + 1;
    const double beta1 = beta[0];
    for (int i = warp; i < l; i += nw) {
        const double* x = X + (size_t)i * NT;
        double nu = 0.0, nv = 0.0;
        for (int k = lane; k < nt; k += 32) {
            double t = x[k] * x[k];
            if (k & 1) nv += t; else nu += t;
        }
        nu = warp_sum(nu);
        nv = warp_sum(nv);
        const double iv = rsqrt(nv);
        for (int k = 2 * lane + 1; k < nt; k += 64) V[(int64_t)i * ldv + (k >> 1)] = x[k] * iv;
        if (U_all) {
            const double iu = rsqrt(nu);
            double* U = U_all + (size_t)b * L * ldu;
            for (int k = 2 * lane; k < nt; k += 64) U[(int64_t)i * ldu + (k >> 1)] = x[k] * iu;
        }
        if (lane == 0) ftil[i] = beta1 * x[0] * rsqrt(nu);
    }
    // f~_{l+1} = beta_1 / |u|, u_1 = 1, log|u_{j+1}| = log|u_j| + log(alpha_j / beta_{j+1})
    // Ls[j] = log|u_{j+1}| for j = 0..l (inclusive prefix sums)
    const bool zero_tail = beta[l] == 0.0;
    for (int j = threadIdx.x; j <= l; j += blockDim.x)
        Ls[j] = (j == 0 || zero_tail) ? 0.0 : log(alpha[j - 1]) - log(beta[j]);
    __syncthreads();
    if (threadIdx.x == 0) {
        // sequential prefix sums (l additions) and log-sum-exp
        double acc = 0.0, mx = 0.0;
        for (int j = 0; j <= l; ++j) {
            acc += Ls[j];
            Ls[j] = acc;
            mx = fmax(mx, acc);
        }
        red[0] = mx;
    }
    __syncthreads();
    const double mx = red[0];
    double part = 0.0;
    for (int j = threadIdx.x; j <= l; j += blockDim.x) part += exp(2.0 * (Ls[j] - mx));
    part = warp_sum(part);
    __syncthreads();
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w];
        double ft = zero_tail ? 0.0 : beta1 * exp(-mx) / sqrt(s);
        ftil[l] = ft;
        if (sigma1_out) sigma1_out[b] = sigma_all[(size_t)b * L];
        if (ftil_last_out) ftil_last_out[b] = ft;
        if (stt && b == 0) {
            stt->scal[SC_FTIL_LAST] = ft;
            stt->scal[SC_SIGMA1] = sigma_all[0];
        }
    }
}

}  // namespace

size_t svd_ws_bytes(int l) { return svd_ws_bytes_batch(l, 1); }

size_t svd_ws_bytes_batch(int L, int B) {
    const size_t NT = 2 * (size_t)L + 1;
    size_t b = 0;
    b += 4 * ws_align(NT * L * 8 * B);            // X, invdp, rp, rm
    b += ws_align((size_t)8 * B);
    return b + 4096;
}

rbf_status launch_projected_svd_batch(rbf_ctx* ctx, ProjDims d, const double* alpha, const double* beta,
                                      double* sigma, double* ftil, double* V, int64_t ldv, void* ws,
                                      double* sigma1_out, double* ftil_last_out, double* U, int64_t ldu) {
    const int L = d.L, B = d.B;
    if (L < 1 || L > SVD_MAX_L)
        return rbf_fail(ctx, RBF_ERR_INVALID, "bidiagonal dimension %d outside [1, %d]", L, SVD_MAX_L);
    const size_t NT = 2 * (size_t)L + 1;
    WsCarve wc(ws);
    double* X = wc.take<double>(NT * L * B);
    double* invdp = wc.take<double>(NT * L * B);
    double* rp = wc.take<double>(NT * L * B);
    double* rm = wc.take<double>(NT * L * B);
    double* bound = wc.take<double>((size_t)B);
    cudaStream_t s = ctx->stream;
    const size_t sh_b = 2 * (size_t)L * sizeof(double);  // also the vectors' e
    const size_t sh_f = ((size_t)L + 1) * sizeof(double);
    if (sh_b > 48 * 1024) {
        RBF_CUDA(ctx, cudaFuncSetAttribute(k_tgk_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_b));
        RBF_CUDA(ctx, cudaFuncSetAttribute(k_tgk_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_b));
    }
    if (sh_f > 48 * 1024)
        RBF_CUDA(ctx, cudaFuncSetAttribute(k_tgk_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_f));
    k_tgk_bisect<<<dim3((L + BS_WARPS - 1) / BS_WARPS, B), BS_WARPS * 32, sh_b, s>>>(d, alpha, beta, sigma, bound);
    RBF_LAUNCHED(ctx, "k_tgk_bisect");
    k_tgk_vectors<<<dim3((L + 31) / 32, B), 32, sh_b, s>>>(d, alpha, beta, sigma, bound, invdp, rp, rm, X);
    RBF_LAUNCHED(ctx, "k_tgk_vectors");
    // at most l / 2 clusters of two or more: one warp each
    const int gy = ((L + 1) / 2 + CL_WARPS - 1) / CL_WARPS;
    if (gy > 65535) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "too many clusters for the grid");
    k_tgk_clusters<<<dim3(B, gy), CL_WARPS * 32, 0, s>>>(d, sigma, ctx->opt.cluster_tol, invdp, rp, X);
    RBF_LAUNCHED(ctx, "k_tgk_clusters");
    k_tgk_finalize<<<B, 256, sh_f, s>>>(d, alpha, beta, X, ftil, V, ldv, B == 1 ? ctx->d_state : nullptr, sigma,
                                        sigma1_out, ftil_last_out, U, ldu);
    RBF_LAUNCHED(ctx, "k_tgk_finalize");
    return RBF_OK;
}

rbf_status launch_projected_svd(rbf_ctx* ctx, const double* alpha, const double* beta, int l,
                                double* sigma, double* ftil, double* V, int64_t ldv, void* ws) {
    if (l < 1 || l > 1023) return rbf_fail(ctx, RBF_ERR_INVALID, "projected dimension %d outside [1, 1023]", l);
    ProjDims d{1, l, l, nullptr};
    return launch_projected_svd_batch(ctx, d, alpha, beta, sigma, ftil, V, ldv, ws, nullptr, nullptr);
}

extern "C" rbf_status rbf_projected_svd(rbf_ctx* ctx, const rbf_gkb_state* st, double* d_sigma,
                                        double* d_ftil, double* d_V, int64_t ldv) {
    RbfRange range_("rbf_projected_svd");
    if (!ctx) return RBF_ERR_INVALID;
    if (!st || !d_sigma || !d_ftil || !d_V) return rbf_fail(ctx, RBF_ERR_INVALID, "NULL argument");
    const int l = st->steps_done;
    if (l < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "state has no completed step");
    if (ldv < l) return rbf_fail(ctx, RBF_ERR_INVALID, "ldv < l");
    RBF_TRY(rbf_ws_reserve(ctx, svd_ws_bytes(l)));
    rbf_timer_start(ctx);
    RBF_TRY(launch_projected_svd(ctx, st->d_alpha, st->d_beta, l, d_sigma, d_ftil, d_V, ldv, ctx->ws));
    ctx->tim.svd_ms = rbf_timer_stop(ctx);
    return RBF_OK;
}
