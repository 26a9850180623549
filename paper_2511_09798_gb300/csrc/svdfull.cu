// Full SVD of the assembled FP64 collocation matrix (Algorithm 3 step 1) and
// the full-SVD methods on top of it: Tikhonov with GCV (Algorithm 3, eqs.
// gcv_svd and tikh_svd_solution) and TSVD (eq. tsvd_solution).
//
// Default: Householder bidiagonalization A = Q_L B Q_R^T in one cooperative
// kernel (per step a left reflector on column k applied to the trailing
// columns and to f, which rides along as an extra column so that g = Q_L^T f
// comes out of the same pass, then a right reflector on row k applied to the
// trailing rows; bounded grid barriers between the phases), then the SVD of
// the bidiagonal through the Golub-Kahan tridiagonal (the projected-SVD
// kernels with C = [B^T; 0]: sigma, V~ = U_B and U~ = V_B), f^ = V~^T g and
// alpha = Q_R (U~ d).
//
// Option svd_method = 1: one-sided (Hestenes) Jacobi (high relative accuracy
// for small singular values, far more work): the columns of W = A are rotated in
// pairs until they are mutually orthogonal (W = U Sigma, V = product of the
// rotations).  One cooperative kernel per sweep: each round pairs the columns
// by the circle method (n/2 disjoint pairs), one CTA per pair: the three dot
// products |w_i|^2, |w_j|^2, w_i.w_j in one pass, the rotation that zeroes
// w_i.w_j applied to w_i, w_j and v_i, v_j; a bounded grid barrier separates
// the rounds.  Sweeps repeat until no pair needed a rotation (|w_i.w_j| <=
// sqrt(n) eps |w_i| |w_j|).  Then sigma_j = |w_j| sorted descending and
// f^ = W^T f / sigma.
//
// Both: numerical rank r = #{sigma_i > N eps sigma_1}, s_perp = sum_{i>r}
// f^_i^2, the GCV grid (Tikhonov) or rank curve (TSVD), the solution alpha.
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

// ---------------------------------------------------------------------------
// Householder bidiagonalization path (n <= 1023)
// ---------------------------------------------------------------------------
constexpr int BT = 256;
constexpr int BW = BT / 32;
// the bidiagonalization kernel runs one CTA per SM of NT threads: 1024 above
// n = 2048, so that enough loads of the trailing matrix are in flight (with 8
// warps per SM the passes over it were bound by load latency: 1.26 -> 0.91 s
// per GCV Tikhonov at n = 4000), 256 below (the per-step block reductions
// over 32 warps cost more than they gain there: 48 -> 59 ms at n = 1000)
constexpr int BIDIAG_BIG_N = 2048;

template <int NW>
__device__ __forceinline__ double block_sum1(double v, double* red) {
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += red[w];
    return t;
}

// Reflector H = I - tau v v^T with v = [1; x_rest * scale] and H x = beta e_1,
// from x_0 and ss = |x_rest|^2 (tau = 0: no reflection needed).
__device__ __forceinline__ void reflector(double x0, double ss, double* sc) {
    if (ss == 0.0) {
        sc[0] = 0.0;
        sc[1] = 0.0;
        sc[2] = x0;
        return;
    }
    const double nrm = sqrt(fma(x0, x0, ss));
    const double beta = x0 >= 0.0 ? -nrm : nrm;
    sc[0] = (beta - x0) / beta;
    sc[1] = 1.0 / (x0 - beta);
    sc[2] = beta;
}

// W column-major n x (n+1) (ld n), the last column f.  On return: dg = diag
// of B, eg = superdiagonal, column n = Q_L^T f, the right reflectors in rows
// k (entries k+2..n-1, unscaled) with taur / scaler.
template <int NT>
__global__ void __launch_bounds__(NT) k_bidiag(double* __restrict__ W, int64_t n, double* __restrict__ dg,
                                               double* __restrict__ eg, double* __restrict__ taur,
                                               double* __restrict__ scaler, rbf_dev_state* __restrict__ stt,
                                               unsigned* __restrict__ bar, int group, long long budget) {
    constexpr int NW = NT / 32;
    __shared__ double red[NW];
    __shared__ double sc[3];
    __shared__ double rp[NW][32];
    __shared__ double rw[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t GW = (int64_t)gridDim.x * NW, gw = (int64_t)blockIdx.x * NW + warp;
    for (int64_t k = 0; k < n; ++k) {
        // left reflector of column k (rows k..n-1), every CTA computes it
        const double* xk = W + k * n + k;
        const int64_t m = n - k;
        double ss = 0.0;
        for (int64_t i = 1 + threadIdx.x; i < m; i += NT) ss = fma(xk[i], xk[i], ss);
        ss = block_sum1<NW>(ss, red);
        if (threadIdx.x == 0) reflector(xk[0], ss, sc);
        __syncthreads();
        const double tau = sc[0], scale = sc[1];
        if (tau != 0.0) {
            for (int64_t j = k + 1 + gw; j <= n; j += GW) {  // warp per trailing column, f included
                double* wj = W + j * n + k;
                const double w0 = wj[0];
                double sd = 0.0, sd1 = 0.0;
                int64_t i = 1 + lane;
                for (; i + 32 < m; i += 64) {
                    sd = fma(xk[i], wj[i], sd);
                    sd1 = fma(xk[i + 32], wj[i + 32], sd1);
                }
                if (i < m) sd = fma(xk[i], wj[i], sd);
                sd = warp_sum(sd + sd1);
                const double t = tau * fma(scale, sd, w0);
                const double ts = t * scale;
                for (int64_t i = 1 + lane; i < m; i += 32) wj[i] = fma(-ts, xk[i], wj[i]);
                if (lane == 0) wj[0] = w0 - t;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) dg[k] = sc[2];
        if (!grid_sync(stt, bar, group, budget)) return;
        if (k == n - 1) break;
        // right reflector of row k (columns k+1..n-1)
        const int64_t m2 = n - k - 1;
        double ss2 = 0.0;
        for (int64_t c = 1 + threadIdx.x; c < m2; c += NT) {
            const double y = W[(k + 1 + c) * n + k];
            ss2 = fma(y, y, ss2);
        }
        ss2 = block_sum1<NW>(ss2, red);
        if (threadIdx.x == 0) reflector(W[(k + 1) * n + k], ss2, sc);
        __syncthreads();
        const double tau2 = sc[0], scale2 = sc[1];
        if (tau2 != 0.0) {
            // blocks of RB rows over the CTAs (RB = 32, 16 or 8: the largest that
            // still gives every CTA a block); lane = (row r, column lane cl), warp
            // q takes the columns c = q CPL + cl, stepping by NW CPL (coalesced
            // along the rows); partial dots combined in shared memory in a fixed
            // order (for RB = 32 one column per warp step, as before)
            const int64_t rows = n - k - 1;
            const int RB = rows >= 32 * (int64_t)gridDim.x ? 32 : (rows >= 16 * (int64_t)gridDim.x ? 16 : 8);
            const int CPL = 32 / RB, CW = NW * CPL;
            const int r = lane % RB, cl = lane / RB;
            const int64_t nblk = (rows + RB - 1) / RB;
            for (int64_t rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
                const int64_t i = k + 1 + rb * RB + r;
                const bool ok = i < n;
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                int64_t c = 1 + warp * CPL + cl;
                for (; c + 3 * CW < m2; c += 4 * CW) {
                    if (ok) {
                        a0 = fma(W[(k + 1 + c) * n + i], W[(k + 1 + c) * n + k], a0);
                        a1 = fma(W[(k + 1 + c + CW) * n + i], W[(k + 1 + c + CW) * n + k], a1);
                        a2 = fma(W[(k + 1 + c + 2 * CW) * n + i], W[(k + 1 + c + 2 * CW) * n + k], a2);
                        a3 = fma(W[(k + 1 + c + 3 * CW) * n + i], W[(k + 1 + c + 3 * CW) * n + k], a3);
                    }
                }
                for (; c < m2; c += CW)
                    if (ok) a0 = fma(W[(k + 1 + c) * n + i], W[(k + 1 + c) * n + k], a0);
                rp[warp][lane] = (a0 + a1) + (a2 + a3);
                __syncthreads();
                if (warp == 0 && lane < RB) {
                    double t = 0.0;
                    for (int q = 0; q < NW; ++q)
                        for (int l = 0; l < CPL; ++l) t += rp[q][l * RB + lane];
                    const int64_t ir = k + 1 + rb * RB + lane;
                    const double x0 = ir < n ? W[(k + 1) * n + ir] : 0.0;
                    rw[lane] = tau2 * fma(scale2, t, x0);  // t_i = tau (u . w_i)
                }
                __syncthreads();
                const double ti = rw[r];
                if (ok) {
                    if (warp == 0 && cl == 0) W[(k + 1) * n + i] -= ti;
                    const double tsi = ti * scale2;
                    for (int64_t cc = 1 + warp * CPL + cl; cc < m2; cc += CW)
                        W[(k + 1 + cc) * n + i] = fma(-tsi, W[(k + 1 + cc) * n + k], W[(k + 1 + cc) * n + i]);
                }
                __syncthreads();
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            eg[k] = sc[2];
            taur[k] = tau2;
            scaler[k] = scale2;
        }
        if (!grid_sync(stt, bar, group, budget)) return;
    }
}

// alpha / beta of C = [B^T; 0] for the tridiagonal SVD: alpha = dg, beta =
// (1, eg, 0); beta_1 only scales f~, which is not used here.
__global__ void k_bidiag_ab(const double* __restrict__ dg, const double* __restrict__ eg, int64_t n,
                            double* __restrict__ alpha, double* __restrict__ beta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) alpha[i] = dg[i];
    if (i <= n) beta[i] = i == 0 ? 1.0 : (i < n ? eg[i - 1] : 0.0);
}

// fhat[i] = V~_i . g  (V~ column-major, ld n; one CTA per i)
__global__ void __launch_bounds__(BT) k_vt_g(const double* __restrict__ Vt, int64_t n, const double* __restrict__ g,
                                             double* __restrict__ fhat) {
    __shared__ double red[BW];
    const double* v = Vt + (int64_t)blockIdx.x * n;
    double a = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += BT) a = fma(v[k], g[k], a);
    a = block_sum1<BW>(a, red);
    if (threadIdx.x == 0) fhat[blockIdx.x] = a;
}

// x[row] = sum_i U~[row][i] d_i over the first n rows of U~ (ld n+1)
__global__ void k_u_d(const double* __restrict__ Ut, int64_t n, const double* __restrict__ d, double* __restrict__ x) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double di = d[i];
        if (di != 0.0) acc = fma(Ut[i * (n + 1) + row], di, acc);
    }
    x[row] = acc;
}

// Z <- Q_R Z, one CTA per column (ld ldz): the right reflectors in reverse order.
__global__ void __launch_bounds__(BT) k_apply_qr(const double* __restrict__ W, int64_t n,
                                                 const double* __restrict__ taur, const double* __restrict__ scaler,
                                                 double* __restrict__ Z, int64_t ldz) {
    __shared__ double red[BW];
    double* z = Z + (int64_t)blockIdx.x * ldz;
    for (int64_t k = n - 2; k >= 0; --k) {
        const double tau = taur[k];
        if (tau == 0.0) continue;
        const double scale = scaler[k];
        const int64_t m2 = n - k - 1;
        const double z0 = z[k + 1];
        double sd = 0.0;
        for (int64_t c = 1 + threadIdx.x; c < m2; c += BT) sd = fma(W[(k + 1 + c) * n + k], z[k + 1 + c], sd);
        sd = block_sum1<BW>(sd, red);
        const double t = tau * fma(scale, sd, z0);
        const double ts = t * scale;
        for (int64_t c = 1 + threadIdx.x; c < m2; c += BT) z[k + 1 + c] = fma(-ts, W[(k + 1 + c) * n + k], z[k + 1 + c]);
        if (threadIdx.x == 0) z[k + 1] = z0 - t;
        __syncthreads();
    }
}

// out[:, k] = V[:, perm k] (column-major)
__global__ void k_gather_cols(const double* __restrict__ V, int64_t n, const int* __restrict__ perm,
                              double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k = blockIdx.y;
    if (i < n) out[k * n + i] = V[(int64_t)perm[k] * n + i];
}

// out[:, k] = U~[0..n-1, k] (drop the last row of U~, ld n+1 -> n)
__global__ void k_copy_ut(const double* __restrict__ Ut, int64_t n, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k = blockIdx.y;
    if (i < n) out[k * n + i] = Ut[k * (n + 1) + i];
}

constexpr int64_t TGK_MAX_N = 8192;

// Result of either path.
struct Fsvd {
    bool tgk;
    int64_t n;
    double *sig, *fhat, *d, *curve, *sperp;
    int* r;
    // Jacobi
    double *W, *V;
    int* perm;
    // bidiagonalization
    double *Wb, *taur, *scaler, *Vt, *Ut;
    int sweeps;
};

int coop_grid(rbf_ctx* ctx, const void* kernel, int threads, int cap, int* group, int* bar_k) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    int G = ctx->sm_count * (occ < 1 ? 1 : occ);
    if (G > cap) G = cap;
    if (G < 1) G = 1;
    int gr = 1;
    while (gr * gr < G) ++gr;
    *group = gr;
    *bar_k = (G + gr - 1) / gr;
    return G;
}

rbf_status fsvd_common_tail(rbf_ctx* ctx, Fsvd* F, const double* f) {
    cudaStream_t s = ctx->stream;
    if (f) {
        k_fsvd_rank<<<1, 32, 0, s>>>(F->sig, F->fhat, F->n, F->r, F->sperp);
        RBF_LAUNCHED(ctx, "k_fsvd_rank");
    }
    return RBF_OK;
}

// Jacobi path
rbf_status fsvd_jacobi(rbf_ctx* ctx, const rbf_operator* op, const double* f, Fsvd* F) {
    const int64_t n = op->n;
    const int np = (int)(n + (n & 1));
    int group, bar_k;
    const int G = coop_grid(ctx, (const void*)k_jacobi_sweep, JT, np / 2, &group, &bar_k);
    const int J = ctx->opt.grid_j;
    const size_t need = 2 * ws_align((size_t)n * n * 8) + 5 * ws_align((size_t)n * 8) +
                        ws_align((size_t)(J > n ? J : n) * 8) + ws_align(8) + ws_align((size_t)n * 4) + ws_align(4) +
                        ws_align((size_t)G * 4) + ws_align((size_t)(bar_k + 2) * BAR_STRIDE * 4) + 4096;
    RBF_TRY(rbf_ws_reserve(ctx, need));
    WsCarve wc(ctx->ws);
    F->tgk = false;
    F->n = n;
    F->W = wc.take<double>((size_t)n * n);
    F->V = wc.take<double>((size_t)n * n);
    double* sig_raw = wc.take<double>((size_t)n);
    F->sig = wc.take<double>((size_t)n);
    F->fhat = wc.take<double>((size_t)n);
    F->d = wc.take<double>((size_t)n);
    F->curve = wc.take<double>((size_t)(J > n ? J : n));
    F->sperp = wc.take<double>(1);
    F->perm = wc.take<int>((size_t)n);
    F->r = wc.take<int>(1);
    int* rotc = wc.take<int>((size_t)G);
    unsigned* bar = wc.take<unsigned>((size_t)(bar_k + 2) * BAR_STRIDE);
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaMemsetAsync(bar, 0, (size_t)(bar_k + 2) * BAR_STRIDE * sizeof(unsigned), s));
    RBF_CUDA(ctx, cudaMemsetAsync(&ctx->d_state->info[IN_ERR], 0, 2 * sizeof(int), s));  // IN_DONE, IN_ERR
    dim3 tb(32, 8), tg((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    k_fsvd_init<<<tg, tb, 0, s>>>((const double*)op->d_A, op->lda, n, F->W, F->V);
    RBF_LAUNCHED(ctx, "k_fsvd_init");
    double tol = sqrt((double)n) * DBL_EPSILON;
    long long budget = ctx->opt.wait_budget;
    std::vector<int> rot((size_t)G);
    int sweeps = 0;
    for (; sweeps < MAX_SWEEPS; ++sweeps) {
        double* Wp = F->W;
        double* Vp = F->V;
        int64_t nn = n;
        int npp = np;
        rbf_dev_state* stt = ctx->d_state;
        int grp = group;
        int* rp = rotc;
        unsigned* bp = bar;
        void* args[] = {&Wp, &Vp, &nn, &npp, &tol, &stt, &bp, &grp, &budget, &rp};
        RBF_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_jacobi_sweep, dim3(G), dim3(JT), args, 0, s));
        ctx->launches++;
        int err = 0;
        RBF_CUDA(ctx, cudaMemcpyAsync(rot.data(), rotc, sizeof(int) * G, cudaMemcpyDeviceToHost, s));
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
    F->sweeps = sweeps;
    k_colnorm<<<(unsigned)n, JT, 0, s>>>(F->W, n, sig_raw);
    RBF_LAUNCHED(ctx, "k_colnorm");
    k_sort_rank<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sig_raw, n, F->perm, F->sig);
    RBF_LAUNCHED(ctx, "k_sort_rank");
    if (f) {
        k_fhat<<<(unsigned)n, JT, 0, s>>>(F->W, n, F->perm, F->sig, f, F->fhat);
        RBF_LAUNCHED(ctx, "k_fhat");
    }
    return fsvd_common_tail(ctx, F, f);
}

// Bidiagonalization path
rbf_status fsvd_bidiag(rbf_ctx* ctx, const rbf_operator* op, const double* f, Fsvd* F) {
    const int64_t n = op->n;
    int group, bar_k;
    const bool big = n > BIDIAG_BIG_N;
    const void* kbid = big ? (const void*)k_bidiag<1024> : (const void*)k_bidiag<256>;
    const int nt = big ? 1024 : 256;
    const int G = coop_grid(ctx, kbid, nt, ctx->sm_count, &group, &bar_k);
    const int J = ctx->opt.grid_j;
    const int L = (int)n;
    const size_t need = ws_align((size_t)n * (n + 1) * 8) + ws_align((size_t)n * n * 8) +
                        ws_align((size_t)(n + 1) * n * 8) + 8 * ws_align((size_t)(n + 2) * 8) +
                        ws_align((size_t)(J > n ? J : n) * 8) + ws_align(8) + ws_align(4) +
                        ws_align((size_t)(bar_k + 2) * BAR_STRIDE * 4) + svd_ws_bytes(L) + 4096;
    RBF_TRY(rbf_ws_reserve(ctx, need));
    WsCarve wc(ctx->ws);
    F->tgk = true;
    F->n = n;
    F->sweeps = 0;
    F->Wb = wc.take<double>((size_t)n * (n + 1));
    F->Vt = wc.take<double>((size_t)n * n);
    F->Ut = wc.take<double>((size_t)(n + 1) * n);
    double* dg = wc.take<double>((size_t)n + 2);
    double* eg = wc.take<double>((size_t)n + 2);
    F->taur = wc.take<double>((size_t)n + 2);
    F->scaler = wc.take<double>((size_t)n + 2);
    double* alpha = wc.take<double>((size_t)n + 2);
    double* beta = wc.take<double>((size_t)n + 2);
    double* ftil = wc.take<double>((size_t)n + 2);
    F->sig = wc.take<double>((size_t)n + 2);
    F->fhat = wc.take<double>((size_t)n + 2);
    F->d = wc.take<double>((size_t)n + 2);
    F->curve = wc.take<double>((size_t)(J > n ? J : n));
    F->sperp = wc.take<double>(1);
    F->r = wc.take<int>(1);
    unsigned* bar = wc.take<unsigned>((size_t)(bar_k + 2) * BAR_STRIDE);
    void* svd = (void*)wc.take<char>(svd_ws_bytes(L));
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaMemsetAsync(bar, 0, (size_t)(bar_k + 2) * BAR_STRIDE * sizeof(unsigned), s));
    RBF_CUDA(ctx, cudaMemsetAsync(&ctx->d_state->info[IN_ERR], 0, 2 * sizeof(int), s));
    RBF_CUDA(ctx, cudaMemsetAsync(F->taur, 0, sizeof(double) * (n + 2), s));
    // W = [A f] column-major (V is only a scratch target of the init kernel here)
    dim3 tb(32, 8), tg((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    k_fsvd_init<<<tg, tb, 0, s>>>((const double*)op->d_A, op->lda, n, F->Wb, F->Vt);
    RBF_LAUNCHED(ctx, "k_fsvd_init");
    if (f) RBF_CUDA(ctx, cudaMemcpyAsync(F->Wb + n * n, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    else RBF_CUDA(ctx, cudaMemsetAsync(F->Wb + n * n, 0, sizeof(double) * n, s));
    {
        double* Wp = F->Wb;
        int64_t nn = n;
        double* dp = dg;
        double* ep = eg;
        double* tp = F->taur;
        double* sp = F->scaler;
        rbf_dev_state* stt = ctx->d_state;
        unsigned* bp = bar;
        int grp = group;
        long long budget = ctx->opt.wait_budget;
        void* args[] = {&Wp, &nn, &dp, &ep, &tp, &sp, &stt, &bp, &grp, &budget};
        RBF_CUDA(ctx, cudaLaunchCooperativeKernel(kbid, dim3(G), dim3(nt), args, 0, s));
        ctx->launches++;
    }
    int err = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&err, &ctx->d_state->info[IN_ERR], sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    if (err) return rbf_fail(ctx, (rbf_status)err, "a bounded grid barrier of the bidiagonalization gave up");
    k_bidiag_ab<<<(unsigned)((n + 256) / 256), 256, 0, s>>>(dg, eg, n, alpha, beta);
    RBF_LAUNCHED(ctx, "k_bidiag_ab");
    ProjDims dd{1, L, L, nullptr};
    RBF_TRY(launch_projected_svd_batch(ctx, dd, alpha, beta, F->sig, ftil, F->Vt, n, svd, nullptr, nullptr, F->Ut,
                                       n + 1));
    if (f) {
        k_vt_g<<<(unsigned)n, BT, 0, s>>>(F->Vt, n, F->Wb + n * n, F->fhat);
        RBF_LAUNCHED(ctx, "k_vt_g");
    }
    return fsvd_common_tail(ctx, F, f);
}

rbf_status fsvd_run(rbf_ctx* ctx, const rbf_operator* op, const double* f, Fsvd* F) {
    const int64_t n = op->n;
    if (op->storage != RBF_ASSEMBLED || op->precision != RBF_FP64 || !op->d_A)
        return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "the full SVD needs an assembled FP64 operator");
    if (n < 2 || n > 8192)
        return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "full SVD for 2 <= n <= 8192 (n = %lld)", (long long)n);
    return (n <= TGK_MAX_N && ctx->opt.svd_method == 0) ? fsvd_bidiag(ctx, op, f, F) : fsvd_jacobi(ctx, op, f, F);
}

// coef = V d
rbf_status fsvd_lift(rbf_ctx* ctx, const Fsvd* F, double* coef) {
    const int64_t n = F->n;
    cudaStream_t s = ctx->stream;
    if (!F->tgk) {
        k_fsvd_lift<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(F->V, n, F->perm, F->d, coef);
        RBF_LAUNCHED(ctx, "k_fsvd_lift");
        return RBF_OK;
    }
    k_u_d<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(F->Ut, n, F->d, coef);
    RBF_LAUNCHED(ctx, "k_u_d");
    k_apply_qr<<<1, BT, 0, s>>>(F->Wb, n, F->taur, F->scaler, coef, n);
    RBF_LAUNCHED(ctx, "k_apply_qr");
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
    RbfRange range_("rbf_svd_full");
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_sigma || (d_fhat && !d_f)) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_svd_full: bad argument");
    Fsvd F;
    RBF_TRY(fsvd_run(ctx, op, d_fhat ? d_f : nullptr, &F));
    const int64_t n = op->n;
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaMemcpyAsync(d_sigma, F.sig, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (d_fhat) RBF_CUDA(ctx, cudaMemcpyAsync(d_fhat, F.fhat, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (d_V) {
        if (F.tgk) {
            k_copy_ut<<<dim3((unsigned)((n + 255) / 256), (unsigned)n), 256, 0, s>>>(F.Ut, n, d_V);
            RBF_LAUNCHED(ctx, "k_copy_ut");
            k_apply_qr<<<(unsigned)n, BT, 0, s>>>(F.Wb, n, F.taur, F.scaler, d_V, n);
            RBF_LAUNCHED(ctx, "k_apply_qr");
        } else {
            k_gather_cols<<<dim3((unsigned)((n + 255) / 256), (unsigned)n), 256, 0, s>>>(F.V, n, F.perm, d_V);
            RBF_LAUNCHED(ctx, "k_gather_cols");
        }
    }
    if (sweeps) *sweeps = F.sweeps;
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    RBF_CUDA(ctx, cudaGetLastError());
    return RBF_OK;
}

extern "C" rbf_status rbf_tikhonov(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int rule,
                                   double lambda_in, double* d_coef, rbf_solve_info* info) {
    RbfRange range_("rbf_tikhonov");
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_f || !d_coef) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_tikhonov: NULL argument");
    if (rule != RBF_GCV && rule != RBF_FIXED) return rbf_fail(ctx, RBF_ERR_INVALID, "rule must be RBF_GCV or RBF_FIXED");
    if (rule == RBF_FIXED && !(lambda_in >= 0.0)) return rbf_fail(ctx, RBF_ERR_INVALID, "fixed lambda must be >= 0");
    Fsvd F;
    RBF_TRY(fsvd_run(ctx, op, d_f, &F));
    const int64_t n = op->n;
    const int J = ctx->opt.grid_j;
    cudaStream_t s = ctx->stream;
    const double tlo = ctx->opt.grid_t_lo, thi = ctx->opt.grid_t_hi;
    if (rule == RBF_GCV) {
        k_fsvd_gcv<<<(J + 127) / 128, 128, 0, s>>>(F.sig, F.fhat, n, F.r, F.sperp, J, tlo, thi, F.curve);
        RBF_LAUNCHED(ctx, "k_fsvd_gcv");
    }
    k_fsvd_choose<<<1, 1024, 0, s>>>(F.curve, J, 0, rule == RBF_FIXED, lambda_in, 0, F.sig, F.fhat, F.r, J, tlo, thi,
                                      F.d, n, ctx->d_state);
    RBF_LAUNCHED(ctx, "k_fsvd_choose");
    RBF_TRY(fsvd_lift(ctx, &F, d_coef));
    int r = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&r, F.r, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_TRY(read_state(ctx));
    if (info) {
        info->lambda = ctx->h_state->scal[SC_LAMBDA];
        info->index = ctx->h_state->info[IN_INDEX];
        info->rank = r;
        info->steps = F.sweeps;
        info->sigma1 = ctx->h_state->scal[SC_SIGMA1];
        info->eta = 0.0;
        info->rho = 0.0;
    }
    return RBF_OK;
}

extern "C" rbf_status rbf_tsvd(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int rank, double* d_coef,
                               rbf_solve_info* info) {
    RbfRange range_("rbf_tsvd");
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_f || !d_coef) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_tsvd: NULL argument");
    if (rank < 0 || rank > op->n) return rbf_fail(ctx, RBF_ERR_INVALID, "rank %d outside [0, n]", rank);
    Fsvd F;
    RBF_TRY(fsvd_run(ctx, op, d_f, &F));
    const int64_t n = op->n;
    cudaStream_t s = ctx->stream;
    if (rank == 0) {
        k_fsvd_gcv_rank<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(F.fhat, n, F.r, F.sperp, F.curve);
        RBF_LAUNCHED(ctx, "k_fsvd_gcv_rank");
    }
    int r = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&r, F.r, sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    const int kmax = (int)(r < n - 1 ? r : n - 1);
    if (rank == 0 && kmax < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "numerical rank 0: no TSVD solution");
    k_fsvd_choose<<<1, 1024, 0, s>>>(F.curve, kmax, 1, rank != 0, 0.0, rank, F.sig, F.fhat, F.r, ctx->opt.grid_j,
                                      ctx->opt.grid_t_lo, ctx->opt.grid_t_hi, F.d, n, ctx->d_state);
    RBF_LAUNCHED(ctx, "k_fsvd_choose");
    RBF_TRY(fsvd_lift(ctx, &F, d_coef));
    RBF_TRY(read_state(ctx));
    if (info) {
        info->lambda = 0.0;
        info->index = -1;
        info->rank = ctx->h_state->info[IN_RANK];
        info->steps = F.sweeps;
        info->sigma1 = ctx->h_state->scal[SC_SIGMA1];
        info->eta = 0.0;
        info->rho = 0.0;
    }
    return RBF_OK;
}
