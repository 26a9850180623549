// Collocation assembly (Sec. 2.1, eqs. H_entries and augmented_system) and
// reconstruction u(X) (eq. u_reconstruction).
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int AS_TN = 256;  // columns per CTA (one per thread)
constexpr int AS_TM = 16;   // rows per CTA

// Entry of A in FP64.  s = r^2 + c^2; interior rows: L Phi = Delta Phi + k^2 Phi
// = (c^2 + s (2 + k^2 s)) s^{-3/2} (since 2 r^2 + 3 c^2 = 2 s + c^2);
// boundary rows: Phi = s^{1/2}.
__device__ __forceinline__ double mq_entry_f64(double dx, double dy, double dz, double c2, double k2,
                                               bool interior) {
    double s = fma(dx, dx, fma(dy, dy, fma(dz, dz, c2)));
    double rs = rsqrt_f64(s);
    if (!interior) return s * rs;
    double poly = fma(s, fma(k2, s, 2.0), c2);
    return (rs * rs) * (rs * poly);
}

__device__ __forceinline__ float mq_entry_f32(float dx, float dy, float dz, float c2, float k2,
                                              bool interior) {
    float s = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, c2)));
    float rs = rsqrtf(s);
    if (!interior) return s * rs;
    float poly = fmaf(s, fmaf(k2, s, 2.0f), c2);
    return (rs * rs) * (rs * poly);
}

template <typename T>
__global__ void __launch_bounds__(AS_TN) k_assemble(const double* __restrict__ X, int64_t n,
                                                    int64_t ni, double c, double k, double scale,
                                                    T* __restrict__ A, int64_t lda) {
    __shared__ double rx[AS_TM], ry[AS_TM], rz[AS_TM];
    const int64_t j = (int64_t)blockIdx.x * AS_TN + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * AS_TM;
    if (threadIdx.x < AS_TM) {
        int64_t i = i0 + threadIdx.x;
        bool ok = i < n;
        rx[threadIdx.x] = ok ? X[i] : 0.0;
        ry[threadIdx.x] = ok ? X[n + i] : 0.0;
        rz[threadIdx.x] = ok ? X[2 * n + i] : 0.0;
    }
    __syncthreads();
    if (j >= n) return;
    const double xj = X[j], yj = X[n + j], zj = X[2 * n + j];
    const double c2 = c * c, k2 = k * k;
    const int rows = (int)min((int64_t)AS_TM, n - i0);
    for (int r = 0; r < rows; ++r) {
        const int64_t i = i0 + r;
        T v;
        if constexpr (sizeof(T) == 8) {
            v = mq_entry_f64(rx[r] - xj, ry[r] - yj, rz[r] - zj, c2, k2, i < ni) * scale;
        } else {
            v = mq_entry_f32((float)rx[r] - (float)xj, (float)ry[r] - (float)yj,
                             (float)rz[r] - (float)zj, (float)c2, (float)k2, i < ni) *
                (float)scale;
        }
        A[i * lda + j] = v;
    }
}

// Partial reconstruction: part[chunk][t] = sum_{j in chunk} coef_j Phi(|P_t - X_j|).
constexpr int EV_T = 128;
__global__ void __launch_bounds__(EV_T) k_evaluate_partial(const double* __restrict__ X, int64_t n,
                                                          const double* __restrict__ coef,
                                                          const double* __restrict__ P, int64_t m,
                                                          double c, double scale, int64_t chunk,
                                                          double* __restrict__ part) {
    __shared__ double sx[EV_T], sy[EV_T], sz[EV_T], sa[EV_T];
    const int64_t t = (int64_t)blockIdx.x * EV_T + threadIdx.x;
    const bool active = t < m;
    const double px = active ? P[t] : 0.0, py = active ? P[m + t] : 0.0, pz = active ? P[2 * m + t] : 0.0;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);
    const double c2 = c * c;
    double acc0 = 0.0, acc1 = 0.0;
    for (int64_t jb = j0; jb < j1; jb += EV_T) {
        __syncthreads();
        int64_t j = jb + threadIdx.x;
        bool ok = j < j1;
        sx[threadIdx.x] = ok ? X[j] : 0.0;
        sy[threadIdx.x] = ok ? X[n + j] : 0.0;
        sz[threadIdx.x] = ok ? X[2 * n + j] : 0.0;
        sa[threadIdx.x] = ok ? coef[j] : 0.0;
        __syncthreads();
        const int cnt = (int)min((int64_t)EV_T, j1 - jb);
        int q = 0;
        for (; q + 1 < cnt; q += 2) {
            double dx0 = px - sx[q], dy0 = py - sy[q], dz0 = pz - sz[q];
            double dx1 = px - sx[q + 1], dy1 = py - sy[q + 1], dz1 = pz - sz[q + 1];
            double s0 = fma(dx0, dx0, fma(dy0, dy0, fma(dz0, dz0, c2)));
            double s1 = fma(dx1, dx1, fma(dy1, dy1, fma(dz1, dz1, c2)));
            acc0 = fma(sa[q], s0 * rsqrt_f64(s0), acc0);
            acc1 = fma(sa[q + 1], s1 * rsqrt_f64(s1), acc1);
        }
        if (q < cnt) {
            double dx0 = px - sx[q], dy0 = py - sy[q], dz0 = pz - sz[q];
            double s0 = fma(dx0, dx0, fma(dy0, dy0, fma(dz0, dz0, c2)));
            acc0 = fma(sa[q], s0 * rsqrt_f64(s0), acc0);
        }
    }
    if (active) part[(int64_t)blockIdx.y * m + t] = (acc0 + acc1) * scale;
}

}  // namespace

rbf_status launch_assemble(rbf_ctx* ctx, const rbf_operator* op) {
    const int64_t n = op->n;
    dim3 grid((unsigned)((n + AS_TN - 1) / AS_TN), (unsigned)((n + AS_TM - 1) / AS_TM));
    if (grid.y > 65535u) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large for assembly grid");
    const double scale = op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0;
    if (op->precision == RBF_FP64)
        k_assemble<double><<<grid, AS_TN, 0, ctx->stream>>>(op->d_nodes, n, op->n_interior, op->c,
                                                            op->k, scale, (double*)op->d_A, op->lda);
    else
        k_assemble<float><<<grid, AS_TN, 0, ctx->stream>>>(op->d_nodes, n, op->n_interior, op->c,
                                                           op->k, scale, (float*)op->d_A, op->lda);
    RBF_LAUNCHED(ctx, "k_assemble");
    return RBF_OK;
}

rbf_status launch_evaluate(rbf_ctx* ctx, const rbf_operator* op, const double* coef,
                           const double* pts, int64_t m, double* u) {
    const int64_t n = op->n;
    const int64_t tiles = (m + EV_T - 1) / EV_T;
    // enough CTAs to occupy every SM's FP64 units: ~8 CTAs per SM in total
    int64_t want = (int64_t)ctx->sm_count * 8;
    int64_t chunks = (want + tiles - 1) / tiles;
    chunks = chunks < 1 ? 1 : chunks;
    int64_t min_chunk = 256;
    if ((n + chunks - 1) / chunks < min_chunk) chunks = (n + min_chunk - 1) / min_chunk;
    if (chunks < 1) chunks = 1;
    if (chunks > 65535) chunks = 65535;
    const int64_t chunk = (n + chunks - 1) / chunks;
    chunks = (n + chunk - 1) / chunk;
    RBF_TRY(rbf_ws_reserve(ctx, ws_align((size_t)chunks * m * sizeof(double))));
    double* part = (double*)ctx->ws;
    const double scale = op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0;
    dim3 grid((unsigned)tiles, (unsigned)chunks);
    k_evaluate_partial<<<grid, EV_T, 0, ctx->stream>>>(op->d_nodes, n, coef, pts, m, op->c, scale,
                                                       chunk, part);
    RBF_LAUNCHED(ctx, "k_evaluate_partial");
    return launch_reduce_partials(ctx, m, (int)chunks, part, u);
}
