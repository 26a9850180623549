// Matrix-free FP32 products with the collocation matrix (mixed precision).
//
// Entry (i, j) is regenerated from the node coordinates on every product (the
// entry formula and the packed f32x2 inner loop are in mf_core.cuh).  Each
// thread keeps MF_R outputs (coordinates, row coefficients and FP64
// accumulators) in registers and streams the summation nodes through shared
// memory; products of one shared tile are summed in FP32 and the tile sum is
// added into the FP64 accumulator.  The summation range is split into chunks
// (grid.y) whose partial sums are reduced deterministically by the consumer.
//   trans = 0: y = A x,   outputs are rows i,    summation over centres j
//   trans = 1: y = A^T x, outputs are centres j, summation over rows i
#include "common.cuh"
#include "internal.h"
#include "mf_core.cuh"

namespace {

constexpr int MF_T = 128;   // threads per CTA
constexpr int MF_R = 4;     // outputs per thread (two f32x2 pairs)
constexpr int MF_S = 256;   // summation nodes per shared tile
constexpr int MF_OUT = MF_T * MF_R;
constexpr int MF_MIN_CTAS = 8;  // resident CTAs per SM the register budget is held to

template <int TRANS>
__global__ void __launch_bounds__(MF_T, MF_MIN_CTAS) k_mf_partial(const double* __restrict__ X, int64_t n,
                                                     int64_t ni, float c2, float k2, double scale,
                                                     const float* __restrict__ x32, int64_t chunk,
                                                     double* __restrict__ part,
                                                     const int* __restrict__ done) {
    if (gkb_done(done)) return;
    constexpr int NP = MF_R / 2;
    __shared__ MfNode tile[MF_S];
    const int64_t obase = (int64_t)blockIdx.x * MF_OUT;
    f2_t OX[NP], OY[NP], OZ[NP], A0[NP], A1[NP], A2[NP];
    double acc[MF_R];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float cx[2], cy[2], cz[2], e0[2], e1[2], e2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t o = obase + threadIdx.x + (2 * p + h) * MF_T;
            const bool ok = o < n;
            cx[h] = ok ? (float)X[o] : 0.f;
            cy[h] = ok ? (float)X[n + o] : 0.f;
            cz[h] = ok ? (float)X[2 * n + o] : 0.f;
            const bool interior = TRANS == 0 && o < ni;
            e0[h] = interior ? c2 : 0.f;
            e1[h] = interior ? 2.f : 0.f;
            e2[h] = interior ? k2 : 1.f;
        }
        OX[p] = f2_pack(cx[0], cx[1]);
        OY[p] = f2_pack(cy[0], cy[1]);
        OZ[p] = f2_pack(cz[0], cz[1]);
        A0[p] = f2_pack(e0[0], e0[1]);
        A1[p] = f2_pack(e1[0], e1[1]);
        A2[p] = f2_pack(e2[0], e2[1]);
        acc[2 * p] = acc[2 * p + 1] = 0.0;
    }
    const f2_t C2 = f2_pack(c2, c2);
    const int64_t s0 = (int64_t)blockIdx.y * chunk;
    const int64_t s1 = min(n, s0 + chunk);
    // For trans = 1 the row type follows the summation index: split at ni.
    for (int seg = 0; seg < (TRANS ? 2 : 1); ++seg) {
        int64_t lo = s0, hi = s1;
        bool bnd = obase >= ni;  // trans = 0: every output row is a Dirichlet row
        if (TRANS) {
            if (seg == 0) {
                hi = min(s1, ni);
                bnd = false;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    A0[p] = C2;
                    A1[p] = f2_pack(2.f, 2.f);
                    A2[p] = f2_pack(k2, k2);
                }
            } else {
                lo = max(s0, ni);
                bnd = true;
            }
            if (hi <= lo) continue;
        }
        for (int64_t tb = lo; tb < hi; tb += MF_S) {
            __syncthreads();
            for (int q = threadIdx.x; q < MF_S; q += MF_T) {
                const int64_t s = tb + q;
                tile[q] = s < hi ? mf_node((float)X[s], (float)X[n + s], (float)X[2 * n + s], x32[s])
                                 : mf_node(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            const int cnt = (int)min((int64_t)MF_S, hi - tb);
            f2_t T[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) T[p] = 0ull;
            if (bnd)
                mf_tile<NP, true>(tile, cnt, OX, OY, OZ, A0, A1, A2, C2, T);
            else
                mf_tile<NP, false>(tile, cnt, OX, OY, OZ, A0, A1, A2, C2, T);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float t0, t1;
                f2_unpack(T[p], t0, t1);
                acc[2 * p] += (double)t0;
                acc[2 * p + 1] += (double)t1;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < MF_R; ++r) {
        const int64_t o = obase + threadIdx.x + r * MF_T;
        if (o < n) part[(int64_t)blockIdx.y * n + o] = acc[r] * scale;
    }
}

// FP64 matrix-free products (RBF_FP64 operators): the same entry formula and
// tiling as the FP32 kernel, in FP64 (s^{-1/2} from an FP32 estimate refined
// to FP64 accuracy) with FP64 accumulators; bound by the FP64 pipe (about 15
// FP64 operations per regenerated entry).
template <int TRANS>
__global__ void __launch_bounds__(MF_T) k_mf_partial_f64(const double* __restrict__ X, int64_t n, int64_t ni,
                                                         double c2, double k2, double scale,
                                                         const double* __restrict__ x, int64_t chunk,
                                                         double* __restrict__ part, const int* __restrict__ done) {
    if (gkb_done(done)) return;
    __shared__ double4 tile[MF_S];
    const int64_t obase = (int64_t)blockIdx.x * MF_OUT;
    double ox[MF_R], oy[MF_R], oz[MF_R], a0[MF_R], a1[MF_R], a2[MF_R], acc[MF_R];
#pragma unroll
    for (int r = 0; r < MF_R; ++r) {
        const int64_t o = obase + threadIdx.x + r * MF_T;
        const bool ok = o < n;
        ox[r] = ok ? X[o] : 0.0;
        oy[r] = ok ? X[n + o] : 0.0;
        oz[r] = ok ? X[2 * n + o] : 0.0;
        const bool interior = TRANS == 0 && o < ni;
        a0[r] = interior ? c2 : 0.0;
        a1[r] = interior ? 2.0 : 0.0;
        a2[r] = interior ? k2 : 1.0;
        acc[r] = 0.0;
    }
    const int64_t s0 = (int64_t)blockIdx.y * chunk;
    const int64_t s1 = min(n, s0 + chunk);
    for (int seg = 0; seg < (TRANS ? 2 : 1); ++seg) {
        int64_t lo = s0, hi = s1;
        if (TRANS) {
            const bool pde = seg == 0;
            if (pde) hi = min(s1, ni);
            else lo = max(s0, ni);
#pragma unroll
            for (int r = 0; r < MF_R; ++r) {
                a0[r] = pde ? c2 : 0.0;
                a1[r] = pde ? 2.0 : 0.0;
                a2[r] = pde ? k2 : 1.0;
            }
            if (hi <= lo) continue;
        }
        for (int64_t tb = lo; tb < hi; tb += MF_S) {
            __syncthreads();
            for (int q = threadIdx.x; q < MF_S; q += MF_T) {
                const int64_t sidx = tb + q;
                tile[q] = sidx < hi ? make_double4(X[sidx], X[n + sidx], X[2 * n + sidx], x[sidx])
                                    : make_double4(0.0, 0.0, 0.0, 0.0);
            }
            __syncthreads();
            const int cnt = (int)min((int64_t)MF_S, hi - tb);
            for (int q = 0; q < cnt; ++q) {
                const double4 nd = tile[q];
#pragma unroll
                for (int r = 0; r < MF_R; ++r) {
                    const double dx = ox[r] - nd.x, dy = oy[r] - nd.y, dz = oz[r] - nd.z;
                    const double s = fma(dx, dx, fma(dy, dy, fma(dz, dz, c2)));
                    const double rs = rsqrt_f64(s);
                    const double g = fma(a0[r], rs * rs, fma(a2[r], s, a1[r]));
                    acc[r] = fma(rs * g, nd.w, acc[r]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < MF_R; ++r) {
        const int64_t o = obase + threadIdx.x + r * MF_T;
        if (o < n) part[(int64_t)blockIdx.y * n + o] = acc[r] * scale;
    }
}

// Resident CTAs per SM of the two product kernels (the smaller), per device.
int mf_occupancy(const rbf_ctx* ctx) {
    static int occ[64] = {0};
    const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
    if (!occ[dev]) {
        int a = 0, b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_mf_partial<0>, MF_T, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mf_partial<1>, MF_T, 0) != cudaSuccess) {
            cudaGetLastError();
            return MF_MIN_CTAS;
        }
        occ[dev] = a < b ? a : b;
        if (occ[dev] < 1) occ[dev] = 1;
    }
    return occ[dev];
}

// Grid: output tiles x summation chunks, with tiles x chunks at most one wave
// of resident CTAs (a second, mostly empty wave would cost a whole CTA time).
void mf_plan(const rbf_ctx* ctx, int64_t n, int64_t* tiles, int* chunks, int64_t* chunk_len) {
    *tiles = (n + MF_OUT - 1) / MF_OUT;
    const int64_t wave = (int64_t)ctx->sm_count * mf_occupancy(ctx);
    int64_t ch = wave / *tiles;
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

rbf_status launch_mf_partial(rbf_ctx* ctx, const rbf_operator* op, int trans, const double* x,
                             const float* x32, double* part, const int* done) {
    int64_t tiles, len;
    int ch;
    mf_plan(ctx, op->n, &tiles, &ch, &len);
    if (tiles > 2147483647LL) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large");
    dim3 grid((unsigned)tiles, (unsigned)ch);
    const double scale = op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0;
    if (op->precision == RBF_FP64) {
        const double c2d = op->c * op->c, k2d = op->k * op->k;
        if (trans)
            k_mf_partial_f64<1><<<grid, MF_T, 0, ctx->stream>>>(op->d_nodes, op->n, op->n_interior, c2d, k2d, scale,
                                                                x, len, part, done);
        else
            k_mf_partial_f64<0><<<grid, MF_T, 0, ctx->stream>>>(op->d_nodes, op->n, op->n_interior, c2d, k2d, scale,
                                                                x, len, part, done);
        RBF_LAUNCHED(ctx, "k_mf_partial_f64");
        return RBF_OK;
    }
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
