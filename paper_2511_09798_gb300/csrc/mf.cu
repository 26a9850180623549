// Matrix-free FP32 products with the collocation matrix (mixed precision).
//
// Entry (i, j) is regenerated from the node coordinates on every product:
// s = |X_i - X_j|^2 + c^2, e = s^{-3/2} P(s) with P(s) = c^2 + s (2 + k^2 s) for
// PDE rows (L Phi = Delta Phi + k^2 Phi) and P(s) = s^2 for Dirichlet rows (Phi),
// i.e. both row types share one polynomial P(s) = a2 s^2 + a1 s + a0 with
// per-row coefficients.  Each thread keeps MF_R outputs (coordinates and FP64
// accumulators) in registers and streams the summation nodes through shared
// memory; products of one shared tile are summed in FP32 and the tile sum is
// added into the FP64 accumulator.  The summation range is split into chunks
// (grid.y) whose partial sums are reduced deterministically by the consumer.
//   trans = 0: y = A x,   outputs are rows i,    summation over centres j
//   trans = 1: y = A^T x, outputs are centres j, summation over rows i
#include "common.cuh"
#include "internal.h"

namespace {

constexpr int MF_T = 128;   // threads per CTA
constexpr int MF_R = 4;     // outputs per thread
constexpr int MF_S = 256;   // summation nodes per shared tile
constexpr int MF_OUT = MF_T * MF_R;

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int TRANS>
__global__ void __launch_bounds__(MF_T) k_mf_partial(const double* __restrict__ X, int64_t n,
                                                     int64_t ni, float c2, float k2, double scale,
                                                     const float* __restrict__ x32, int64_t chunk,
                                                     double* __restrict__ part,
                                                     const int* __restrict__ done) {
    if (gkb_done(done)) return;
    __shared__ float4 tile[MF_S];
    const int64_t obase = (int64_t)blockIdx.x * MF_OUT;
    float ox[MF_R], oy[MF_R], oz[MF_R], a2[MF_R], a1[MF_R], a0[MF_R];
    double acc[MF_R];
#pragma unroll
    for (int r = 0; r < MF_R; ++r) {
        const int64_t o = obase + threadIdx.x + r * MF_T;
        const bool ok = o < n;
        ox[r] = ok ? (float)X[o] : 0.f;
        oy[r] = ok ? (float)X[n + o] : 0.f;
        oz[r] = ok ? (float)X[2 * n + o] : 0.f;
        const bool interior = TRANS == 0 && o < ni;
        a2[r] = interior ? k2 : 1.f;
        a1[r] = interior ? 2.f : 0.f;
        a0[r] = interior ? c2 : 0.f;
        acc[r] = 0.0;
    }
    const int64_t s0 = (int64_t)blockIdx.y * chunk;
    const int64_t s1 = min(n, s0 + chunk);
    // For trans = 1 the row type follows the summation index: split at ni.
    for (int seg = 0; seg < (TRANS ? 2 : 1); ++seg) {
        int64_t lo = s0, hi = s1;
        float b2 = 0.f, b1 = 0.f, b0 = 0.f;
        if (TRANS) {
            if (seg == 0) { hi = min(s1, ni); b2 = k2; b1 = 2.f; b0 = c2; }
            else { lo = max(s0, ni); b2 = 1.f; b1 = 0.f; b0 = 0.f; }
            if (hi <= lo) continue;
        }
        for (int64_t tb = lo; tb < hi; tb += MF_S) {
            __syncthreads();
            for (int q = threadIdx.x; q < MF_S; q += MF_T) {
                const int64_t s = tb + q;
                float4 v;
                if (s < hi) {
                    v.x = (float)X[s];
                    v.y = (float)X[n + s];
                    v.z = (float)X[2 * n + s];
                    v.w = x32[s];
                } else {
                    v = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                tile[q] = v;
            }
            __syncthreads();
            const int cnt = (int)min((int64_t)MF_S, hi - tb);
            float t[MF_R];
#pragma unroll
            for (int r = 0; r < MF_R; ++r) t[r] = 0.f;
#pragma unroll 4
            for (int q = 0; q < cnt; ++q) {
                const float4 cq = tile[q];
#pragma unroll
                for (int r = 0; r < MF_R; ++r) {
                    const float dx = ox[r] - cq.x, dy = oy[r] - cq.y, dz = oz[r] - cq.z;
                    const float s = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, c2)));
                    const float rs = rsqrt_approx(s);
                    const float P = TRANS ? fmaf(s, fmaf(b2, s, b1), b0) : fmaf(s, fmaf(a2[r], s, a1[r]), a0[r]);
                    const float rs3 = (rs * rs) * rs;
                    t[r] = fmaf(rs3 * P, cq.w, t[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < MF_R; ++r) acc[r] += (double)t[r];
        }
    }
#pragma unroll
    for (int r = 0; r < MF_R; ++r) {
        const int64_t o = obase + threadIdx.x + r * MF_T;
        if (o < n) part[(int64_t)blockIdx.y * n + o] = acc[r] * scale;
    }
}

void mf_plan(const rbf_ctx* ctx, int64_t n, int64_t* tiles, int* chunks, int64_t* chunk_len) {
    *tiles = (n + MF_OUT - 1) / MF_OUT;
    int64_t want = (int64_t)ctx->sm_count * 8;
    int64_t ch = (want + *tiles - 1) / *tiles;
    if (ch < 1) ch = 1;
    int64_t max_ch = (n + MF_S - 1) / MF_S;  // at least one shared tile per chunk
    if (ch > max_ch) ch = max_ch;
    if (ch > 65535) ch = 65535;
    *chunk_len = (n + ch - 1) / ch;
    *chunks = (int)((n + *chunk_len - 1) / *chunk_len);
}

}  // namespace

int mf_chunks(const rbf_ctx* ctx, const rbf_operator* op) {
    int64_t tiles, len;
    int ch;
    mf_plan(ctx, op->n, &tiles, &ch, &len);
    return ch;
}

size_t mf_ws_bytes(const rbf_ctx* ctx, int64_t n) {
    int64_t tiles, len;
    int ch;
    mf_plan(ctx, n, &tiles, &ch, &len);
    return ws_align((size_t)ch * n * sizeof(double));
}

rbf_status launch_mf_partial(rbf_ctx* ctx, const rbf_operator* op, int trans, const float* x32,
                             double* part, const int* done) {
    if (op->precision != RBF_MIXED)
        return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "matrix-free products are FP32 (RBF_MIXED)");
    int64_t tiles, len;
    int ch;
    mf_plan(ctx, op->n, &tiles, &ch, &len);
    if (tiles > 2147483647LL) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large");
    dim3 grid((unsigned)tiles, (unsigned)ch);
    const double scale = op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0;
    const float c2 = (float)(op->c * op->c), k2 = (float)(op->k * op->k);
    if (trans)
        k_mf_partial<1><<<grid, MF_T, 0, ctx->stream>>>(op->d_nodes, op->n, op->n_interior, c2, k2,
                                                        scale, x32, len, part, done);
    else
        k_mf_partial<0><<<grid, MF_T, 0, ctx->stream>>>(op->d_nodes, op->n, op->n_interior, c2, k2,
                                                        scale, x32, len, part, done);
    RBF_LAUNCHED(ctx, "k_mf_partial");
    return RBF_OK;
}
