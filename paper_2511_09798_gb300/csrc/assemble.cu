// Collocation assembly (Sec. 2.1, eqs. H_entries and augmented_system) and
// reconstruction u(X) (eq. u_reconstruction).
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int AS_TN = 256;  // columns per CTA (one per thread)
constexpr int AS_TM = 16;   // rows per CTA

// Entry of A.  s = r^2 + c^2; interior rows: L Phi = Delta Phi + k^2 Phi
// = (c^2 + s (2 + k^2 s)) s^{-3/2} (since 2 r^2 + 3 c^2 = 2 s + c^2);
// boundary rows: Phi = s^{1/2}.
__device__ __forceinline__ double lphi_from(double s, double rs, double c2, double k2) {
    const double poly = fma(s, fma(k2, s, 2.0), c2);
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

// FP32 assembly (mixed precision): one column per thread, AS_TM rows per CTA.
// The coordinates are rounded to FP32 once per row (shared memory) and once
// per column (registers), not once per entry: the conversions run at the
// FP64 rate.
__global__ void __launch_bounds__(AS_TN) k_assemble_f32(const double* __restrict__ X, int64_t n, int64_t ni,
                                                        double c, double k, double scale, float* __restrict__ A,
                                                        int64_t lda) {
    __shared__ float rx[AS_TM], ry[AS_TM], rz[AS_TM];
    const int64_t j = (int64_t)blockIdx.x * AS_TN + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * AS_TM;
    if (threadIdx.x < AS_TM) {
        int64_t i = i0 + threadIdx.x;
        bool ok = i < n;
        rx[threadIdx.x] = ok ? (float)X[i] : 0.f;
        ry[threadIdx.x] = ok ? (float)X[n + i] : 0.f;
        rz[threadIdx.x] = ok ? (float)X[2 * n + i] : 0.f;
    }
    __syncthreads();
    if (j >= n) return;
    const float xj = (float)X[j], yj = (float)X[n + j], zj = (float)X[2 * n + j];
    const float c2 = (float)(c * c), k2 = (float)(k * k), sc = (float)scale;
    const int rows = (int)min((int64_t)AS_TM, n - i0);
    for (int r = 0; r < rows; ++r) {
        const int64_t i = i0 + r;
        A[i * lda + j] = mq_entry_f32(rx[r] - xj, ry[r] - yj, rz[r] - zj, c2, k2, i < ni) * sc;
    }
}

// FP64 assembly by pairs of 32-row tiles.  The entries (i, j) and (j, i)
// share s = |X_i - X_j|^2 + c^2 and 1/sqrt(s) (the squared differences do not
// change sign), and are equal whenever rows i and j are of the same kind, so
// one CTA per tile pair (I <= J) computes s and 1/sqrt(s) once for the 32 x 32
// node pairs, writes tile (I, J) row by row and tile (J, I) through a
// shared-memory transpose (coalesced stores in both).  CTAs below the
// diagonal return at once.
constexpr int SY_T = 32;     // tile edge
constexpr int SY_ROWS = 8;   // thread rows per CTA

// NM operators that share the nodes and c (and so s and 1/sqrt(s)) but differ
// in k are assembled together: Phi, 1/s and the distances once, the k-dependent
// polynomial of L Phi per matrix (same operations, in the same order, as for
// one matrix).
template <int NM>
struct AsmOut {
    double* A[NM];
    int64_t lda[NM];
    double k2[NM];
};

template <int NM>
__global__ void __launch_bounds__(SY_T * SY_ROWS) k_assemble_sym_f64(const double* __restrict__ X, int64_t n,
                                                                      int64_t ni, double c, double scale,
                                                                      AsmOut<NM> o) {
    __shared__ double tr[NM][SY_T][SY_T + 1];
    __shared__ double pi[3][SY_T], pj[3][SY_T];
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi > bj) return;
    const int tx = threadIdx.x % SY_T, ty = threadIdx.x / SY_T;
    const int64_t I0 = (int64_t)bi * SY_T, J0 = (int64_t)bj * SY_T;
    if (threadIdx.x < SY_T) {
        const int64_t i = I0 + threadIdx.x, j = J0 + threadIdx.x;
        for (int d = 0; d < 3; ++d) {
            pi[d][threadIdx.x] = i < n ? X[d * n + i] : 0.0;
            pj[d][threadIdx.x] = j < n ? X[d * n + j] : 0.0;
        }
    }
    __syncthreads();
    const double c2 = c * c;
    const int64_t j = J0 + tx;
    const bool jint = j < ni;
    const bool scaled = scale != 1.0;
#pragma unroll
    for (int rr = 0; rr < SY_T / SY_ROWS; ++rr) {
        const int li = ty + SY_ROWS * rr;
        const int64_t i = I0 + li;
        double eji[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) eji[m] = 0.0;
        if (i < n && j < n) {
            const double dx = pi[0][li] - pj[0][tx], dy = pi[1][li] - pj[1][tx], dz = pi[2][li] - pj[2][tx];
            const double s = fma(dx, dx, fma(dy, dy, fma(dz, dz, c2)));
            const double rs = rsqrt_f64(s);
            const bool iint = i < ni;
            const double phi = s * rs;
            const bool need_l = iint || jint;
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const double lp = need_l ? lphi_from(s, rs, c2, o.k2[m]) : 0.0;
                double eij = iint ? lp : phi;
                double e2 = jint == iint ? eij : (jint ? lp : phi);
                if (scaled) {
                    eij *= scale;
                    e2 *= scale;
                }
                if (RBF_IN_RANGE(j, o.lda[m])) o.A[m][i * o.lda[m] + j] = eij;
                eji[m] = e2;
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) tr[m][li][tx] = eji[m];
    }
    if (bi == bj) return;
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < SY_T / SY_ROWS; ++rr) {
        const int lj = ty + SY_ROWS * rr;
        const int64_t jr = J0 + lj, ic = I0 + tx;
        if (jr < n && ic < n)
#pragma unroll
            for (int m = 0; m < NM; ++m)
                if (RBF_IN_RANGE(ic, o.lda[m])) o.A[m][jr * o.lda[m] + ic] = tr[m][tx][lj];
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
    if (op->precision == RBF_FP64) {
        const int64_t nt = (n + SY_T - 1) / SY_T;
        if (nt > 65535) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large for assembly grid");
        AsmOut<1> o{{(double*)op->d_A}, {op->lda}, {op->k * op->k}};
        k_assemble_sym_f64<1><<<dim3((unsigned)nt, (unsigned)nt), SY_T * SY_ROWS, 0, ctx->stream>>>(
            op->d_nodes, n, op->n_interior, op->c, scale, o);
        RBF_LAUNCHED(ctx, "k_assemble_sym_f64");
        return RBF_OK;
    }
    k_assemble_f32<<<grid, AS_TN, 0, ctx->stream>>>(op->d_nodes, n, op->n_interior, op->c, op->k, scale,
                                                    (float*)op->d_A, op->lda);
    RBF_LAUNCHED(ctx, "k_assemble_f32");
    return RBF_OK;
}

bool assemble_pairable(const rbf_operator* a, const rbf_operator* b) {
    return a->storage == RBF_ASSEMBLED && b->storage == RBF_ASSEMBLED && a->precision == RBF_FP64 &&
           b->precision == RBF_FP64 && a->d_nodes == b->d_nodes && a->n == b->n && a->n_interior == b->n_interior &&
           a->c == b->c && a->form == b->form && a->d_A != b->d_A;
}

rbf_status launch_assemble_pair(rbf_ctx* ctx, const rbf_operator* a, const rbf_operator* b) {
    if (!assemble_pairable(a, b)) return rbf_fail(ctx, RBF_ERR_INTERNAL, "operators cannot be assembled together");
    const int64_t n = a->n;
    const int64_t nt = (n + SY_T - 1) / SY_T;
    if (nt > 65535) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large for assembly grid");
    const double scale = a->form == RBF_FORM_EPS ? 1.0 / a->c : 1.0;
    AsmOut<2> o{{(double*)a->d_A, (double*)b->d_A}, {a->lda, b->lda}, {a->k * a->k, b->k * b->k}};
    k_assemble_sym_f64<2><<<dim3((unsigned)nt, (unsigned)nt), SY_T * SY_ROWS, 0, ctx->stream>>>(
        a->d_nodes, n, a->n_interior, a->c, scale, o);
    RBF_LAUNCHED(ctx, "k_assemble_sym_f64<2>");
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

RBF_CHECK_READER(assemble)
