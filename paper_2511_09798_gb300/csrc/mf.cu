// Matrix-free products with the collocation matrix.
//
// FP32 entries (mixed precision): tile pairs.  Rows and columns of A are the
// same node list, s_ij = |X_i - X_j|^2 + c^2 = s_ji, and an entry depends on
// its row's type only (L Phi for PDE rows, Phi for Dirichlet rows), so the
// PDE x PDE and Dirichlet x Dirichlet blocks are symmetric.  The nodes are cut
// into nb blocks of B; CTA (I, J), I < J, evaluates s and s^{-1/2} once per
// node pair (i in I, j in J) and feeds both A_ij and A_ji (one value when the
// two rows have the same type): y_i += A_ij x_j and y_j += A_ji x_i for y = A x,
// the mirror for y = A^T x.  Diagonal tiles (I == I) take every ordered pair
// once.  Partial sums: the contributions of tile (I, J) to the outputs of block
// I go to slot J, those to the outputs of block J to slot I, so every output
// receives exactly one value in each of the nb slots and the consumer sums
// the slots in a fixed order (deterministic, no atomics).
//
// Inside a CTA the tile's rows sit in registers (R per lane, f32x2 pairs) and
// its four warps split the columns; a warp stages 32 columns in shared memory
// and runs over them together (one broadcast read per column).  The column
// sums (A_ji x_i over the warp's rows) leave each step as one FP32 value per
// lane and are added over the lanes through a padded shared array after 32
// columns.  FP32 runs: a row sum covers the B <= 256 columns of the tile, a
// column sum its B rows; each then goes to FP64 (the node coordinates come
// rounded to FP32 from the caller, converted once per GKB run).
//
// FP64 operators: one output per thread, summation nodes streamed through
// shared memory in chunks (grid.y), partials per chunk.
//   trans = 0: y = A x,   trans = 1: y = A^T x
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "mf_core.cuh"

namespace {

// ---- FP32 tile-pair kernel (the tile product itself is in mf_core.cuh) ----
// Tile t of the nb (nb + 1) / 2 tiles (I, J), I <= J.  The FP32 square root
// estimates the row; the integer loops correct it (the FP64 pipe is slow).
__device__ __forceinline__ void ms_tile(int64_t t, int64_t nb, int64_t& I, int64_t& J) {
    const int64_t u = nb * (nb + 1) / 2 - 1 - t;
    int64_t r = (int64_t)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
    if (r < 0) r = 0;
    while ((r + 1) * (r + 2) / 2 <= u) ++r;
    while (r > 0 && r * (r + 1) / 2 > u) --r;
    I = nb - 1 - r;
    J = nb - 1 - (u - r * (r + 1) / 2);
}

// One tile per CTA, tiles in the order of ms_tile.
template <int TRANS, int R>
__global__ void __launch_bounds__(MS_W * 32) k_mf_sym(const float* __restrict__ X, int64_t n, int64_t ni, float c2,
                                                    float k2, double scale, const float* __restrict__ x32,
                                                    int64_t nb, double* __restrict__ part,
                                                    const int* __restrict__ done) {
    if (gkb_done(done)) return;
    int64_t I, J;
    ms_tile(blockIdx.x, nb, I, J);
    ms_tile_product<TRANS, R>(X, n, ni, c2, k2, scale, x32, I, J, part);
}

// Fold the nb slots (rows G .. G + nb - 1 of the partial buffer) into G
// groups of k consecutive slots (rows 0 .. G - 1), each group summed in order;
// one thread per (output, group).
__global__ void k_ms_fold(double* __restrict__ part, int64_t n, int nb, int k, const int* __restrict__ done) {
    if (gkb_done(done)) return;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int g = blockIdx.y, G = gridDim.y;
    const int s1 = min(nb, (g + 1) * k);
    double acc = 0.0;
    for (int s = g * k; s < s1; ++s) acc += part[(int64_t)(G + s) * n + o];
    part[(int64_t)g * n + o] = acc;
}

constexpr int MF_T = 128;   // FP64 kernel: threads per CTA
constexpr int MF_R = 4;     // outputs per thread
constexpr int MF_S = 256;   // summation nodes per shared tile
constexpr int MF_OUT = MF_T * MF_R;

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

// Resident CTAs per SM of a kernel pair (the smaller), cached per device.
template <typename K0, typename K1>
int pair_occupancy(int* cache, const rbf_ctx* ctx, K0 k0, K1 k1, int threads, int fallback) {
    const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
    if (!cache[dev]) {
        int a = 0, b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k0, threads, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k1, threads, 0) != cudaSuccess) {
            cudaGetLastError();
            return fallback;
        }
        cache[dev] = a < b ? a : b;
        if (cache[dev] < 1) cache[dev] = 1;
    }
    return cache[dev];
}

// FP64 kernel grid: output tiles x summation chunks, with tiles x chunks at
// most one wave of resident CTAs (a second, mostly empty wave would cost a
// whole CTA time).
void mf_plan(const rbf_ctx* ctx, int64_t n, int64_t* tiles, int* chunks, int64_t* chunk_len) {
    static int occ[64] = {0};
    *tiles = (n + MF_OUT - 1) / MF_OUT;
    const int64_t wave =
        (int64_t)ctx->sm_count * pair_occupancy(occ, ctx, k_mf_partial_f64<0>, k_mf_partial_f64<1>, MF_T, 4);
    int64_t ch = wave / *tiles;
    if (ch < 1) ch = 1;
    int64_t max_ch = (n + MF_S - 1) / MF_S;  // at least one shared tile per chunk
    if (ch > max_ch) ch = max_ch;
    if (ch > 65535) ch = 65535;
    *chunk_len = (n + ch - 1) / ch;
    *chunks = (int)((n + *chunk_len - 1) / *chunk_len);
}

// FP32 tile-pair grid: blocks of 256 (8 rows per lane) once their tiles fill
// the resident CTAs at least once, else blocks of 128 (4 rows per lane, four
// times as many tiles).
// The consumer of the partials (the GKB half-step) stages slots x rows-per-SM
// doubles in shared memory: above 12288 of them (96 KB) the nb slots are first
// folded into G <= 12288 / rows-per-SM groups (at least 8, at most 128).  The
// fold costs a launch and a pass over the slots (13 us of a 106 us product at
// n = 20000, where 79 slots now fit unfolded).
struct MsPlan {
    int R;
    int64_t nb, tiles;
    int k, G;  // slots per group, groups (G = nb, k = 1: no fold)
};
MsPlan ms_plan(const rbf_ctx* ctx, int64_t n) {
    static int occ[64] = {0};
    MsPlan pl{};
    const int64_t nb8 = (n + 255) / 256;
    const int64_t t8 = nb8 * (nb8 + 1) / 2;
    const int64_t wave = (int64_t)ctx->sm_count * pair_occupancy(occ, ctx, k_mf_sym<0, 8>, k_mf_sym<1, 8>, MS_W * 32, 4);
    if (t8 >= wave) {
        pl.R = 8;
        pl.nb = nb8;
    } else {
        pl.R = 4;
        pl.nb = (n + 127) / 128;
    }
    pl.tiles = pl.nb * (pl.nb + 1) / 2;
    const int64_t sm = ctx->sm_count > 0 ? ctx->sm_count : 1;
    const int64_t rows = (n + sm - 1) / sm;
    int64_t gmax = 12288 / (rows > 0 ? rows : 1);
    gmax = gmax < 8 ? 8 : (gmax > 128 ? 128 : gmax);
    if (pl.nb <= gmax) {
        pl.k = 1;
        pl.G = (int)pl.nb;
    } else {
        pl.k = (int)((pl.nb + gmax - 1) / gmax);
        pl.G = (int)((pl.nb + pl.k - 1) / pl.k);
    }
    return pl;
}

}  // namespace

int mf_chunks(const rbf_ctx* ctx, const rbf_operator* op) {
    if (op->precision != RBF_FP64) return ms_plan(ctx, op->n).G;
    int64_t tiles, len;
    int ch;
    mf_plan(ctx, op->n, &tiles, &ch, &len);
    return ch;
}

int mf_part_rows(const rbf_ctx* ctx, const rbf_operator* op) {
    if (op->precision != RBF_FP64) {
        const MsPlan pl = ms_plan(ctx, op->n);
        return (int)pl.nb + (pl.k > 1 ? pl.G : 0);
    }
    return mf_chunks(ctx, op);
}

size_t mf_ws_bytes(const rbf_ctx* ctx, int64_t n) {
    int64_t tiles, len;
    int ch;
    mf_plan(ctx, n, &tiles, &ch, &len);
    const MsPlan pl = ms_plan(ctx, n);
    const int64_t rows = pl.nb + (pl.k > 1 ? pl.G : 0);
    return ws_align((size_t)(rows > ch ? rows : ch) * n * sizeof(double));
}

rbf_status launch_mf_partial(rbf_ctx* ctx, const rbf_operator* op, int trans, const double* x,
                             const float* x32, const float* X32, double* part, const int* done) {
    const double scale = op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0;
    if (op->precision == RBF_FP64) {
        int64_t tiles, len;
        int ch;
        mf_plan(ctx, op->n, &tiles, &ch, &len);
        if (tiles > 2147483647LL) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large");
        dim3 grid((unsigned)tiles, (unsigned)ch);
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
    const MsPlan pl = ms_plan(ctx, op->n);
    if (pl.tiles > 2147483647LL) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large");
    if (!X32 || !x32) return rbf_fail(ctx, RBF_ERR_INTERNAL, "FP32 product without its FP32 inputs");
    const float c2 = (float)(op->c * op->c), k2 = (float)(op->k * op->k);
    const unsigned grid = (unsigned)pl.tiles;
    const int64_t n = op->n, ni = op->n_interior;
    double* slots = part + (pl.k > 1 ? (int64_t)pl.G * n : 0);  // folded: slots after the G group rows
    if (pl.R == 8) {
        if (trans) k_mf_sym<1, 8><<<grid, MS_W * 32, 0, ctx->stream>>>(X32, n, ni, c2, k2, scale, x32, pl.nb, slots, done);
        else k_mf_sym<0, 8><<<grid, MS_W * 32, 0, ctx->stream>>>(X32, n, ni, c2, k2, scale, x32, pl.nb, slots, done);
    } else {
        if (trans) k_mf_sym<1, 4><<<grid, MS_W * 32, 0, ctx->stream>>>(X32, n, ni, c2, k2, scale, x32, pl.nb, slots, done);
        else k_mf_sym<0, 4><<<grid, MS_W * 32, 0, ctx->stream>>>(X32, n, ni, c2, k2, scale, x32, pl.nb, slots, done);
    }
    RBF_LAUNCHED(ctx, "k_mf_sym");
    if (pl.k > 1) {
        k_ms_fold<<<dim3((unsigned)((n + 255) / 256), (unsigned)pl.G), 256, 0, ctx->stream>>>(part, n, (int)pl.nb, pl.k,
                                                                                             done);
        RBF_LAUNCHED(ctx, "k_ms_fold");
    }
    return RBF_OK;
}
