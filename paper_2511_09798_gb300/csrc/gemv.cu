// Assembled matrix-vector products of Algorithm 1: p = A z (row-major GEMV;
// FP64: an equal share of the entries per warp, partials per row piece; FP32:
// balanced (row, column-segment) units per warp, partials per segment) and
// r = A^T w (GEMV^T by row chunks); every partial sum is reduced in a fixed
// order by the consumer, so results are deterministic.
//
// A is streamed once per product with 16-byte vector loads (evict-first), the
// input vector is read through L1.  FP64 operators use FP64 FMAs (on GB300 the
// FP64 pipe, 2 FMA/clk/SM, and not HBM bounds this product).  FP32 (mixed)
// operators multiply in FP32 and add short FP32 runs of products into FP64
// accumulators.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int GN_THREADS = 256;  // 8 warps, one (row, segment) unit per warp at a time
constexpr int GT_THREADS = 256;
constexpr int GT_MAX_CHUNK_ROWS = 4096;

__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }

// ---------------------------------------------------------------------------
// FP64 A x by the flat split of the matrix (flat_bound): each row piece of a
// warp is reduced across the warp and written to part[slot][row], slot = w
// minus the first warp that touches the row; the warp holding the end of a
// row writes zeros into the row's remaining slots, so part[0 .. chunks-1][row]
// always sum to (A x)_row.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(GN_THREADS) k_gemv_flat_f64(
    const double* __restrict__ A, int64_t lda, int64_t n, const double* __restrict__ x, int64_t W, int chunks,
    double* __restrict__ part, const int* __restrict__ done) {
    if (gkb_done(done)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (GN_THREADS / 32) + warp;
    if (w >= W) return;
    const int64_t e0 = flat_bound(n, W, w), e1 = flat_bound(n, W, w + 1);
    if (e1 <= e0) return;
    const int64_t r0 = e0 / n, r1 = (e1 - 1) / n;
    for (int64_t r = r0; r <= r1; ++r) {
        const int64_t cs = r == r0 ? e0 - r * n : 0;
        const int64_t ce = r == r1 ? e1 - r * n : n;
        int64_t wf = w;  // first warp of the row
        while (wf > 0 && flat_bound(n, W, wf) > r * n) --wf;
        const int slot = (int)(w - wf);
        const double2* __restrict__ row = reinterpret_cast<const double2*>(A + r * lda + cs);
        const double2* __restrict__ xv = reinterpret_cast<const double2*>(x + cs);
        const int64_t nvec = (ce - cs) >> 1;
        // piece lengths are multiples of 128 columns except at a row's end, so
        // every lane is busy in all but the row's last loads
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int64_t v = lane;
        for (; v + 96 < nvec; v += 128) {
            double2 m0 = ld_stream(row + v), m1 = ld_stream(row + v + 32);
            double2 m2 = ld_stream(row + v + 64), m3 = ld_stream(row + v + 96);
            double2 x0 = __ldg(xv + v), x1 = __ldg(xv + v + 32);
            double2 x2 = __ldg(xv + v + 64), x3 = __ldg(xv + v + 96);
            a0 = fma(m0.x, x0.x, a0); a0 = fma(m0.y, x0.y, a0);
            a1 = fma(m1.x, x1.x, a1); a1 = fma(m1.y, x1.y, a1);
            a2 = fma(m2.x, x2.x, a2); a2 = fma(m2.y, x2.y, a2);
            a3 = fma(m3.x, x3.x, a3); a3 = fma(m3.y, x3.y, a3);
        }
        a0 += a2;
        a1 += a3;
        for (; v < nvec; v += 32) {
            double2 m0 = ld_stream(row + v), x0 = __ldg(xv + v);
            a0 = fma(m0.x, x0.x, a0); a0 = fma(m0.y, x0.y, a0);
        }
        if (((ce - cs) & 1) && lane == 0) a1 = fma(A[r * lda + ce - 1], __ldg(x + ce - 1), a1);
        const double acc = warp_sum(a0 + a1);
        if (lane == 0 && RBF_IN_RANGE(slot, chunks)) {
            part[(int64_t)slot * n + r] = acc;
            if (ce == n)
                for (int s2 = slot + 1; s2 < chunks; ++s2) part[(int64_t)s2 * n + r] = 0.0;
        }
    }
}

// FP32 (mixed) version: products of one float4 quad group summed in FP32,
// each group added into the FP64 accumulator; segments start on multiples of
// 4 columns (16-byte aligned float4 loads).
__global__ void __launch_bounds__(GN_THREADS) k_gemv_nseg_f32(
    const float* __restrict__ A, int64_t lda, int64_t n, const float* __restrict__ x32, int S,
    int64_t seglen, double* __restrict__ part, const int* __restrict__ done) {
    if (gkb_done(done)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (GN_THREADS / 32);
    const int64_t w = (int64_t)blockIdx.x * (GN_THREADS / 32) + warp;
    const int64_t U = n * S;
    const int64_t u0 = U * w / W, u1 = U * (w + 1) / W;
    for (int64_t u = u0; u < u1; ++u) {
        const int64_t i = u / S;
        const int g = (int)(u - i * S);
        const int64_t c0 = (int64_t)g * seglen;
        const int64_t c1 = min(n, c0 + seglen);
        const float4* __restrict__ row = reinterpret_cast<const float4*>(A + i * lda + c0);
        const float4* __restrict__ xv = reinterpret_cast<const float4*>(x32 + c0);
        const int64_t nvec = (c1 - c0) >> 2;
        double acc = 0.0;
        int64_t v = lane;
        for (; v + 96 < nvec; v += 128) {
            float4 m0 = ld_stream(row + v), m1 = ld_stream(row + v + 32);
            float4 m2 = ld_stream(row + v + 64), m3 = ld_stream(row + v + 96);
            float4 x0 = __ldg(xv + v), x1 = __ldg(xv + v + 32);
            float4 x2 = __ldg(xv + v + 64), x3 = __ldg(xv + v + 96);
            float s0 = m0.x * x0.x, s1 = m1.x * x1.x, s2 = m2.x * x2.x, s3 = m3.x * x3.x;
            s0 = fmaf(m0.y, x0.y, s0); s1 = fmaf(m1.y, x1.y, s1); s2 = fmaf(m2.y, x2.y, s2); s3 = fmaf(m3.y, x3.y, s3);
            s0 = fmaf(m0.z, x0.z, s0); s1 = fmaf(m1.z, x1.z, s1); s2 = fmaf(m2.z, x2.z, s2); s3 = fmaf(m3.z, x3.z, s3);
            s0 = fmaf(m0.w, x0.w, s0); s1 = fmaf(m1.w, x1.w, s1); s2 = fmaf(m2.w, x2.w, s2); s3 = fmaf(m3.w, x3.w, s3);
            acc += (double)((s0 + s1) + (s2 + s3));
        }
        for (; v < nvec; v += 32) {
            float4 m0 = ld_stream(row + v), x0 = __ldg(xv + v);
            float s0 = m0.x * x0.x;
            s0 = fmaf(m0.y, x0.y, s0); s0 = fmaf(m0.z, x0.z, s0); s0 = fmaf(m0.w, x0.w, s0);
            acc += (double)s0;
        }
        for (int64_t c = c0 + nvec * 4 + lane; c < c1; c += 32) acc += (double)(A[i * lda + c] * x32[c]);
        acc = warp_sum(acc);
        if (lane == 0) part[(int64_t)g * n + i] = acc;
    }
}

// ---------------------------------------------------------------------------
// part[q][c] = sum_{i in row chunk q} A_ic x_i for the columns of this CTA's
// panel; 8 rows of A are loaded before their 16 FMAs (8 independent pairs of
// accumulators), which keeps enough loads in flight to feed the FP64 pipe.
// ---------------------------------------------------------------------------
constexpr int GT_UNROLL = 8;
__global__ void __launch_bounds__(GT_THREADS) k_gemv_t_f64(
    const double* __restrict__ A, int64_t lda, int64_t n, const double* __restrict__ x,
    int panel_cols, int chunks, double* __restrict__ part, const int* __restrict__ done) {
    if (gkb_done(done)) return;
    __shared__ double xs[GT_MAX_CHUNK_ROWS];
    const int q = blockIdx.x % chunks;
    const int pnl = blockIdx.x / chunks;
    const int64_t i0 = n * (int64_t)q / chunks;  // balanced row chunks
    int64_t i1 = n * (int64_t)(q + 1) / chunks;
    if (!RBF_IN_RANGE(i1 - i0, GT_MAX_CHUNK_ROWS + 1)) i1 = i0 + GT_MAX_CHUNK_ROWS;  // the x slab in shared memory
    for (int64_t i = i0 + threadIdx.x; i < i1; i += GT_THREADS) xs[i - i0] = x[i];
    __syncthreads();
    const int64_t c = (int64_t)pnl * panel_cols + 2 * threadIdx.x;
    if (c >= n || i1 <= i0) {
        if (c < n) {
            part[(int64_t)q * n + c] = 0.0;
            if (c + 1 < n) part[(int64_t)q * n + c + 1] = 0.0;
        }
        return;
    }
    const double* __restrict__ base = A + i0 * lda + c;
    // 8 rows of loads in flight, 4 accumulator pairs (rows u and u + 4 share
    // one): the combine at the end costs 6 adds per column pair
    constexpr int GT_ACC = GT_UNROLL / 2;
    double ax[GT_ACC], ay[GT_ACC];
#pragma unroll
    for (int u = 0; u < GT_ACC; ++u) ax[u] = ay[u] = 0.0;
    const int64_t rows = i1 - i0;
    int64_t r = 0;
    for (; r + GT_UNROLL - 1 < rows; r += GT_UNROLL) {
        double2 m[GT_UNROLL];
#pragma unroll
        for (int u = 0; u < GT_UNROLL; ++u) m[u] = ld_stream(reinterpret_cast<const double2*>(base + (r + u) * lda));
#pragma unroll
        for (int u = 0; u < GT_UNROLL; ++u) {
            ax[u % GT_ACC] = fma(m[u].x, xs[r + u], ax[u % GT_ACC]);
            ay[u % GT_ACC] = fma(m[u].y, xs[r + u], ay[u % GT_ACC]);
        }
    }
    for (; r < rows; ++r) {
        double2 m0 = ld_stream(reinterpret_cast<const double2*>(base + r * lda));
        ax[0] = fma(m0.x, xs[r], ax[0]);
        ay[0] = fma(m0.y, xs[r], ay[0]);
    }
    const double sx = (ax[0] + ax[1]) + (ax[2] + ax[3]);
    const double sy = (ay[0] + ay[1]) + (ay[2] + ay[3]);
    part[(int64_t)q * n + c] = sx;
    if (c + 1 < n) part[(int64_t)q * n + c + 1] = sy;
}

__global__ void __launch_bounds__(GT_THREADS) k_gemv_t_f32(
    const float* __restrict__ A, int64_t lda, int64_t n, const float* __restrict__ x32,
    int panel_cols, int chunks, double* __restrict__ part, const int* __restrict__ done) {
    if (gkb_done(done)) return;
    __shared__ float xs[GT_MAX_CHUNK_ROWS];
    const int q = blockIdx.x % chunks;
    const int pnl = blockIdx.x / chunks;
    const int64_t i0 = n * (int64_t)q / chunks;  // balanced row chunks
    const int64_t i1 = n * (int64_t)(q + 1) / chunks;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += GT_THREADS) xs[i - i0] = x32[i];
    __syncthreads();
    const int64_t c = (int64_t)pnl * panel_cols + 4 * threadIdx.x;
    if (c >= n) return;
    const float* __restrict__ base = A + i0 * lda + c;
    double d0 = 0, d1 = 0, d2 = 0, d3 = 0;
    const int64_t rows = i1 - i0;
    int64_t r = 0;
    for (; r + 7 < rows; r += 8) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float4 m = ld_stream(reinterpret_cast<const float4*>(base + (r + u) * lda));
            float xv = xs[r + u];
            s0 = fmaf(m.x, xv, s0); s1 = fmaf(m.y, xv, s1); s2 = fmaf(m.z, xv, s2); s3 = fmaf(m.w, xv, s3);
        }
        d0 += (double)s0; d1 += (double)s1; d2 += (double)s2; d3 += (double)s3;
    }
    for (; r < rows; ++r) {
        float4 m = ld_stream(reinterpret_cast<const float4*>(base + r * lda));
        float xv = xs[r];
        d0 += (double)(m.x * xv); d1 += (double)(m.y * xv); d2 += (double)(m.z * xv); d3 += (double)(m.w * xv);
    }
    double* out = part + (int64_t)q * n + c;
    out[0] = d0;
    if (c + 1 < n) out[1] = d1;
    if (c + 2 < n) out[2] = d2;
    if (c + 3 < n) out[3] = d3;
}

__global__ void k_reduce_partials(int64_t n, int chunks, const double* __restrict__ part,
                                  double* __restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int q = 0; q < chunks; ++q) s += part[(int64_t)q * n + i];
    y[i] = s;
}

// y_i = scale * (sum of the FP32 slots of row i), added in slot order by a
// compensated (Neumaier) FP32 sum carried to FP64 as hi + lo.
__global__ void k_reduce_slots_f32(int64_t n, int chunks, const float* __restrict__ part, double scale,
                                   double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float hi = 0.f, lo = 0.f;
    for (int q = 0; q < chunks; ++q) {
        const float t = part[(int64_t)q * n + i];
        const float sm = hi + t;
        lo += fabsf(hi) >= fabsf(t) ? (hi - sm) + t : (t - sm) + hi;
        hi = sm;
    }
    y[i] = ((double)hi + (double)lo) * scale;
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}

}  // namespace

static void plan_t_sms(int sm_count, int64_t n, int vec, int* panel_cols, int* panels, int* chunks) {
    *panel_cols = GT_THREADS * vec;
    *panels = (int)((n + *panel_cols - 1) / *panel_cols);
    const int slots = sm_count * 4;  // 4 CTAs of 256 threads per SM
    int q = slots / *panels;
    if (q < 1) q = 1;
    // at least 8 rows per chunk, at most GT_MAX_CHUNK_ROWS
    int64_t max_chunks = (n + 7) / 8;
    if (q > max_chunks) q = (int)max_chunks;
    int64_t min_chunks = (n + GT_MAX_CHUNK_ROWS - 1) / GT_MAX_CHUNK_ROWS;
    if (q < min_chunks) q = (int)min_chunks;
    *chunks = q;
}

void plan_t(const rbf_ctx* ctx, int64_t n, int vec, int* panel_cols, int* panels, int* chunks) {
    plan_t_sms(ctx->sm_count, n, vec, panel_cols, panels, chunks);
}

size_t gemv_ws_bytes(const rbf_ctx* ctx, int64_t n) {
    int pc, pn, ch;
    plan_t(ctx, n, 2, &pc, &pn, &ch);
    int pc4, pn4, ch4;
    plan_t(ctx, n, 4, &pc4, &pn4, &ch4);
    int c = ch > ch4 ? ch : ch4;
    if (c < 8) c = 8;  // partial-sum rows of the FP64 A x (at most 8)
    return ws_align((size_t)c * n * sizeof(double)) + ws_align((size_t)n * sizeof(float));
}

int gemv_t_chunks(const rbf_ctx* ctx, const rbf_operator* op) {
    int pc, pn, ch;
    plan_t(ctx, op->n, op->precision == RBF_FP64 ? 2 : 4, &pc, &pn, &ch);
    return ch;
}

static int gemv_n_occupancy(const rbf_ctx* ctx, bool fp64) {
    static int occ[2][64] = {{0}};
    const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
    int& o = occ[fp64 ? 0 : 1][dev];
    if (!o) {
        int a = 0;
        const cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_gemv_flat_f64, GN_THREADS, 0)
                                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_gemv_nseg_f32, GN_THREADS, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            a = 4;
        }
        o = a < 1 ? 1 : a;
    }
    return o;
}

// FP64 A x (flat split): W active warps, at most one wave of resident CTAs,
// at least 256 entries per warp, and few enough warps that no row is split
// into more than 8 pieces (the partial-sum rows the workspace provides).  A
// row of n entries meets at most ceil(n / (per - 2)) + 1 warp ranges, per =
// floor(n^2 / W) (each boundary is rounded down by at most one entry).
void flat_split_plan(int64_t n, int64_t Wmax, int64_t* W_out, int* chunks) {
    const int64_t e = n * n;
    int64_t W = Wmax;
    if (W > e / 256) W = e / 256;
    if (W < 1) W = 1;
    // a warp owns at least per - FLAT_ALIGN entries (each bound is rounded down
    // by less than FLAT_ALIGN), so a row meets at most this many warp ranges
    auto pieces = [&](int64_t w) -> int64_t {
        if (w <= 1) return 1;
        const int64_t per = e / w;
        if (per <= FLAT_ALIGN) return n;  // never taken: W <= e / 256
        return (n + per - FLAT_ALIGN - 1) / (per - FLAT_ALIGN) + 1;
    };
    while (W > 1 && pieces(W) > 8) --W;
    *W_out = W;
    *chunks = (int)pieces(W);
}

static void gemv_flat_plan(const rbf_ctx* ctx, int64_t n, int* grid, int64_t* W_out, int* chunks) {
    flat_split_plan(n, (int64_t)ctx->sm_count * gemv_n_occupancy(ctx, true) * (GN_THREADS / 32), W_out, chunks);
    *grid = (int)((*W_out + GN_THREADS / 32 - 1) / (GN_THREADS / 32));
}

// FP32 A x: grid = one wave of resident CTAs; S column segments per row chosen
// so that the n S units divide as evenly as possible over the grid's warps
// (efficiency x / ceil(x) with x = n S / warps), segments of >= 256 columns.
static void gemv_nseg_plan(const rbf_ctx* ctx, int64_t n, int* grid, int* S, int64_t* seglen) {
    int64_t g = (int64_t)ctx->sm_count * gemv_n_occupancy(ctx, false);
    const int64_t rows_min = (n + 7) / 8;
    if (g > rows_min) g = rows_min;
    if (g < 1) g = 1;
    const double W = (double)g * (GN_THREADS / 32);
    int best = 1;
    double best_eff = 0.0;
    for (int s = 1; s <= 8; ++s) {
        if (s > 1 && n / s < 256) break;
        const double xu = (double)n * s / W;
        const double eff = xu / ceil(xu);
        if (eff > best_eff + 1e-3) {
            best_eff = eff;
            best = s;
        }
    }
    int64_t len = (n + best - 1) / best;
    len = (len + 3) / 4 * 4;  // segments start on 16-byte boundaries
    *grid = (int)g;
    *S = (int)((n + len - 1) / len);
    *seglen = len;
}

int gemv_n_chunks(const rbf_ctx* ctx, const rbf_operator* op) {
    int g, S;
    if (op->precision == RBF_FP64) {
        int64_t W;
        gemv_flat_plan(ctx, op->n, &g, &W, &S);
        return S;
    }
    int64_t len;
    gemv_nseg_plan(ctx, op->n, &g, &S, &len);
    return S;
}

rbf_status launch_gemv_n(rbf_ctx* ctx, const rbf_operator* op, const double* x, const float* x32, double* part,
                         const int* done) {
    int g, S;
    if (op->precision == RBF_FP64) {
        int64_t W;
        gemv_flat_plan(ctx, op->n, &g, &W, &S);
        k_gemv_flat_f64<<<g, GN_THREADS, 0, ctx->stream>>>((const double*)op->d_A, op->lda, op->n, x, W, S, part,
                                                           done);
        RBF_LAUNCHED(ctx, "k_gemv_flat_f64");
    } else {
        int64_t len;
        gemv_nseg_plan(ctx, op->n, &g, &S, &len);
        k_gemv_nseg_f32<<<g, GN_THREADS, 0, ctx->stream>>>((const float*)op->d_A, op->lda, op->n, x32, S, len, part,
                                                           done);
        RBF_LAUNCHED(ctx, "k_gemv_nseg_f32");
    }
    return RBF_OK;
}

rbf_status launch_gemv_t_partial(rbf_ctx* ctx, const rbf_operator* op, const double* x,
                                 const float* x32, double* part, const int* done) {
    int pc, pn, ch;
    if (op->precision == RBF_FP64) {
        plan_t(ctx, op->n, 2, &pc, &pn, &ch);
        k_gemv_t_f64<<<pn * ch, GT_THREADS, 0, ctx->stream>>>((const double*)op->d_A, op->lda, op->n,
                                                              x, pc, ch, part, done);
        RBF_LAUNCHED(ctx, "k_gemv_t_f64");
    } else {
        plan_t(ctx, op->n, 4, &pc, &pn, &ch);
        k_gemv_t_f32<<<pn * ch, GT_THREADS, 0, ctx->stream>>>((const float*)op->d_A, op->lda, op->n,
                                                              x32, pc, ch, part, done);
        RBF_LAUNCHED(ctx, "k_gemv_t_f32");
    }
    return RBF_OK;
}

rbf_status launch_reduce_partials(rbf_ctx* ctx, int64_t n, int chunks, const double* part, double* y) {
    k_reduce_partials<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, chunks, part, y);
    RBF_LAUNCHED(ctx, "k_reduce_partials");
    return RBF_OK;
}

rbf_status launch_reduce_slots_f32(rbf_ctx* ctx, int64_t n, int chunks, const float* part, double scale, double* y) {
    k_reduce_slots_f32<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, chunks, part, scale, y);
    RBF_LAUNCHED(ctx, "k_reduce_slots_f32");
    return RBF_OK;
}

rbf_status launch_to_f32(rbf_ctx* ctx, int64_t n, const double* x, float* y, cudaStream_t s) {
    k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s ? s : ctx->stream>>>(n, x, y);
    RBF_LAUNCHED(ctx, "k_to_f32");
    return RBF_OK;
}

extern "C" rbf_status rbf_matvec(rbf_ctx* ctx, const rbf_operator* op, int trans, const double* d_x,
                                 double* d_y) {
    RbfRange range_("rbf_matvec");
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_x || !d_y) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_matvec: NULL argument");
    const int64_t n = op->n;
    if (op->storage == RBF_MATRIX_FREE) {
        RBF_TRY(rbf_ws_reserve(ctx, mf_ws_bytes(ctx, n) + ws_align((size_t)n * sizeof(float)) +
                                        ws_align((size_t)3 * n * sizeof(float))));
        WsCarve wc(ctx->ws);
        float* x32 = wc.take<float>((size_t)n);
        float* X32 = wc.take<float>((size_t)3 * n);
        double* part = wc.take<double>((size_t)mf_part_rows(ctx, op) * n);
        if (op->precision == RBF_MIXED) {
            RBF_TRY(launch_to_f32(ctx, n, d_x, x32));
            RBF_TRY(launch_to_f32(ctx, 3 * n, op->d_nodes, X32));
        }
        RBF_TRY(launch_mf_partial(ctx, op, trans, d_x, x32, X32, part, nullptr));
        if (mf_slots_f32(ctx, op))
            return launch_reduce_slots_f32(ctx, n, mf_chunks(ctx, op), (const float*)part,
                                           op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0, d_y);
        return launch_reduce_partials(ctx, n, mf_chunks(ctx, op), part, d_y);
    }
    RBF_TRY(rbf_ws_reserve(ctx, gemv_ws_bytes(ctx, n)));
    WsCarve wc(ctx->ws);
    const int ch = gemv_t_chunks(ctx, op);
    double* part = wc.take<double>((size_t)ch * n);
    float* x32 = wc.take<float>((size_t)n);
    if (op->precision == RBF_MIXED) RBF_TRY(launch_to_f32(ctx, n, d_x, x32));
    if (trans == 0) {
        const int S = gemv_n_chunks(ctx, op);
        if (S == 1) return launch_gemv_n(ctx, op, d_x, x32, d_y, nullptr);
        RBF_TRY(launch_gemv_n(ctx, op, d_x, x32, part, nullptr));
        return launch_reduce_partials(ctx, n, S, part, d_y);
    }
    RBF_TRY(launch_gemv_t_partial(ctx, op, d_x, x32, part, nullptr));
    return launch_reduce_partials(ctx, n, ch, part, d_y);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP64 product y = A^T x.
//
// Callers that cannot allocate device memory -- for example code whose device
// memory is reserved up front by another allocator, or a latency-critical loop
// in which cudaMalloc / cudaFree (which may synchronise the whole device) are not
// allowed -- use this entry point.  Its partial sums live in the file-scope
// device array below instead of a context workspace.  The array is part of the
// loaded module: every GPU on which the library is used holds these 8 MiB until
// the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_partials[RBF_NOALLOC_SCRATCH_DOUBLES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
int g_noalloc_sms[NOALLOC_MAX_DEVICES] = {};
}  // namespace

extern "C" rbf_status rbf_matvec_t_noalloc(const double* d_A, int64_t lda, int64_t n, const double* d_x,
                                           double* d_y, void* cuda_stream) {
    if (!d_A || !d_x || !d_y || n <= 0 || lda < n || (lda & 1) || ((uintptr_t)d_A & 15u))
        return RBF_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return RBF_ERR_CUDA;
    double* scratch = nullptr;
    int sms = 0;
    {
        // one-time set-up per device, with that device current: the host-side
        // name of the array is not a device address, so take its address here
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess) return RBF_ERR_CUDA;
            if (cudaDeviceGetAttribute(&g_noalloc_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return RBF_ERR_CUDA;
            g_noalloc_ptr[dev] = (double*)p;
        }
        scratch = g_noalloc_ptr[dev];
        sms = g_noalloc_sms[dev];
    }
    int pc, pn, ch;
    plan_t_sms(sms, n, 2, &pc, &pn, &ch);
    // fit the partial sums into the static array: fewer row chunks if needed
    const int64_t max_chunks = RBF_NOALLOC_SCRATCH_DOUBLES / n;
    const int64_t min_chunks = (n + GT_MAX_CHUNK_ROWS - 1) / GT_MAX_CHUNK_ROWS;
    if (max_chunks < min_chunks) return RBF_ERR_INVALID;  // n beyond the scratch limit
    if (ch > max_chunks) ch = (int)max_chunks;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // an error left pending by earlier, unrelated work is reported (and left in
    // place for its owner) instead of being cleared and blamed on these launches
    if (cudaPeekAtLastError() != cudaSuccess) return RBF_ERR_CUDA;
    // every (chunk, column) partial is written before it is read: nothing to clear
    k_gemv_t_f64<<<pn * ch, GT_THREADS, 0, s>>>(d_A, lda, n, d_x, pc, ch, scratch, nullptr);
    if (cudaGetLastError() != cudaSuccess) return RBF_ERR_CUDA;
    k_reduce_partials<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, ch, scratch, d_y);
    if (cudaGetLastError() != cudaSuccess) return RBF_ERR_CUDA;
    return RBF_OK;
}

RBF_CHECK_READER(gemv)
