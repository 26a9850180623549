// Matrix-free products with the collocation matrix, by tile pairs.
//
// Rows and columns of A are the same node list, s_ij = |X_i - X_j|^2 + c^2 =
// s_ji, and an entry depends on its row's type only (L Phi for PDE rows, Phi for Dirichlet rows), so the
// PDE x PDE and Dirichlet x Dirichlet blocks are symmetric.  The nodes are cut
// into nb blocks of B; CTA (I, J), I < J, evaluates s and s^{-1/2} once per
// node pair (i in I, j in J) and feeds both A_ij and A_ji (one value when the
// two rows have the same type): y_i += A_ij x_j and y_j += A_ji x_i for y = A x,
// the mirror for y = A^T x.  Diagonal tiles (I == J) take every ordered pair
// once.  Partial sums: the contributions of tile (I, J) to the outputs of block
// I go to slot J, those to the outputs of block J to slot I, so every output
// receives exactly one value in each of the nb slots and the consumer sums
// the slots in a fixed order (deterministic, no atomics).
//
// FP32 entries (mixed precision; the tile product is in mf_core.cuh): inside a
// CTA the tile's rows sit in registers (R per lane, f32x2 pairs) and
// its four warps split the columns; a warp stages 32 columns in shared memory
// and runs over them together (one broadcast read per column).  The column
// sums (A_ji x_i over the warp's rows) leave each step as one FP32 value per
// lane and are added over the lanes through a padded shared array after 32
// columns.  FP32 runs: a row sum covers the B <= 256 columns of the tile, a
// column sum its B rows; each then goes to FP64 (the node coordinates come
// rounded to FP32 from the caller, converted once per GKB run).
//
// FP64 operators: the same tiles in FP64 scalars (k_mf_sym_f64).
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

// One tile per CTA, tiles in the order of ms_tile.  Without a fold the nb
// slots hold the FP32 runs themselves (SlotT float; the consumer adds them with
// a compensated FP32 sum and applies scale); when the half-step would stage
// too many slots they are FP64 (run times scale), written after G group rows
// and folded into them (k_ms_fold).
template <int TRANS, int R, typename SlotT>
__global__ void __launch_bounds__(MS_W * 32) k_mf_sym(const float* __restrict__ X, int64_t n, int64_t ni, float c2,
                                                    float k2, double scale, const float* __restrict__ x32,
                                                    int64_t nb, SlotT* __restrict__ part,
                                                    const int* __restrict__ done) {
    if (gkb_done(done)) return;
    int64_t I, J;
    ms_tile(blockIdx.x, nb, I, J);
    if (!RBF_IN_RANGE(J, nb) || !RBF_IN_RANGE(I, J + 1)) return;  // a tile of the triangle: slots I, J < nb
    ms_tile_product<TRANS, R, SlotT>(X, n, ni, c2, k2, scale, x32, I, J, part);
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

// ---- FP64 tile-pair kernel (RBF_FP64 operators) ----
// The same tiles, slots and entry formula as the FP32 kernel, in FP64 scalars
// (s^{-1/2}: an FP32 estimate refined to FP64 accuracy): R rows per lane, the
// four warps of a CTA split the tile's 32 R columns, 32 columns per step
// group staged as double4 (x, y, z, input value).  Column sums leave each step
// as one FP64 value per lane (colpart) and are added over the lanes after 32
// columns; row sums over the warps at the end.  Everything is FP64.
constexpr int MD_R = 4;  // rows per lane: blocks of 128 nodes

template <int TRANS, bool SYM, int RT, int CT>
__device__ __forceinline__ void md_cols(const double4* __restrict__ cols, double (*colpart)[33], int lane,
                                        const double* OX, const double* OY, const double* OZ, const double* XI,
                                        unsigned imask, double c2, double k2, int64_t cb, int64_t ni, double* T) {
    constexpr bool useR = SYM || TRANS == 0;
    constexpr bool useC = SYM || TRANS == 1;
    constexpr bool needL = (useR && RT != MS_BND) || (useC && CT != MS_BND);
    constexpr bool needP = (useR && RT != MS_INT) || (useC && CT != MS_INT);
#pragma unroll 2
    for (int q = 0; q < 32; ++q) {
        const double4 nd = cols[q];
        const bool cint = CT == MS_INT || (CT == MS_MIX && cb + q < ni);
        double CA = 0.0;
#pragma unroll
        for (int r = 0; r < MD_R; ++r) {
            const double dx = OX[r] - nd.x, dy = OY[r] - nd.y, dz = OZ[r] - nd.z;
            const double s = fma(dx, dx, fma(dy, dy, fma(dz, dz, c2)));
            const double rs = rsqrt_f64(s);
            double eL = 0.0, eP = 0.0;
            if constexpr (needL) eL = rs * fma(c2, rs * rs, fma(k2, s, 2.0));
            if constexpr (needP) eP = rs * s;
            const double eR = RT == MS_INT ? eL : (RT == MS_BND ? eP : (((imask >> r) & 1u) ? eL : eP));
            const double eC = cint ? eL : eP;
            T[r] = fma(TRANS == 0 ? eR : eC, nd.w, T[r]);
            if constexpr (SYM) CA = fma(TRANS == 0 ? eC : eR, XI[r], CA);
        }
        if constexpr (SYM) colpart[q][lane] = CA;
    }
}

template <int TRANS, bool SYM>
__device__ __forceinline__ void md_dispatch(int rt, int ct, const double4* cols, double (*colpart)[33], int lane,
                                            const double* OX, const double* OY, const double* OZ, const double* XI,
                                            unsigned imask, double c2, double k2, int64_t cb, int64_t ni, double* T) {
    if (!SYM && TRANS == 0) ct = MS_INT;
    if (!SYM && TRANS == 1) rt = MS_INT;
#define MD_CASE(R_, C_)                                                                                    \
    case R_ * 3 + C_:                                                                                      \
        md_cols<TRANS, SYM, R_, C_>(cols, colpart, lane, OX, OY, OZ, XI, imask, c2, k2, cb, ni, T);          \
        break;
    switch (rt * 3 + ct) {
        MD_CASE(MS_INT, MS_INT)
        MD_CASE(MS_INT, MS_BND)
        MD_CASE(MS_INT, MS_MIX)
        MD_CASE(MS_BND, MS_INT)
        MD_CASE(MS_BND, MS_BND)
        MD_CASE(MS_BND, MS_MIX)
        MD_CASE(MS_MIX, MS_INT)
        MD_CASE(MS_MIX, MS_BND)
        MD_CASE(MS_MIX, MS_MIX)
        default: break;
    }
#undef MD_CASE
}

template <int TRANS>
__global__ void __launch_bounds__(MS_W * 32) k_mf_sym_f64(const double* __restrict__ X, int64_t n, int64_t ni,
                                                        double c2, double k2, double scale,
                                                        const double* __restrict__ x, int64_t nb,
                                                        double* __restrict__ part, const int* __restrict__ done) {
    if (gkb_done(done)) return;
    constexpr int B = 32 * MD_R, CW = B / MS_W;
    static_assert(CW % 32 == 0, "a warp takes whole groups of 32 columns");
    __shared__ double4 cols[MS_W][32];
    __shared__ double colpart[MS_W][32][33];
    __shared__ double own[MS_W][MD_R][32];
    int64_t I, J;
    ms_tile(blockIdx.x, nb, I, J);
    if (!RBF_IN_RANGE(J, nb) || !RBF_IN_RANGE(I, J + 1)) return;  // a tile of the triangle: slots I, J < nb
    const bool sym = I != J;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = I * B, col0 = J * B;
    const int rt = ms_type(row0, row0 + B, ni);
    double OX[MD_R], OY[MD_R], OZ[MD_R], XI[MD_R], T[MD_R];
    unsigned imask = 0;
#pragma unroll
    for (int r = 0; r < MD_R; ++r) {
        const int64_t i = row0 + lane + 32 * r;
        const bool ok = i < n;
        OX[r] = ok ? X[i] : 0.0;
        OY[r] = ok ? X[n + i] : 0.0;
        OZ[r] = ok ? X[2 * n + i] : 0.0;
        XI[r] = ok ? x[i] : 0.0;
        T[r] = 0.0;
        if (i < ni) imask |= 1u << r;
    }
    for (int g = 0; g < CW / 32; ++g) {
        const int64_t cb = col0 + warp * CW + g * 32;
        {
            const int64_t j = cb + lane;
            const bool ok = j < n;
            cols[warp][lane] = ok ? make_double4(X[j], X[n + j], X[2 * n + j], x[j]) : make_double4(0.0, 0.0, 0.0, 0.0);
        }
        __syncwarp();
        const int ct = ms_type(cb, cb + 32, ni);
        if (sym)
            md_dispatch<TRANS, true>(rt, ct, cols[warp], colpart[warp], lane, OX, OY, OZ, XI, imask, c2, k2, cb, ni, T);
        else
            md_dispatch<TRANS, false>(rt, ct, cols[warp], colpart[warp], lane, OX, OY, OZ, XI, imask, c2, k2, cb, ni, T);
        __syncwarp();
        if (sym) {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int m = 0; m < 32; ++m) v[m & 3] += colpart[warp][lane][m];
            const int64_t j = cb + lane;
            if (j < n) part[I * n + j] = ((v[0] + v[1]) + (v[2] + v[3])) * scale;
            __syncwarp();
        }
    }
#pragma unroll
    for (int r = 0; r < MD_R; ++r) own[warp][r][lane] = T[r];
    __syncthreads();
    for (int e = threadIdx.x; e < B; e += MS_W * 32) {
        const int r = e >> 5, l = e & 31;
        const int64_t i = row0 + l + 32 * r;
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < MS_W; ++w) acc += own[w][r][l];
        if (i < n) part[J * n + i] = acc * scale;
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

// Tile-pair grid.  FP32: blocks of 256 (8 rows per lane) once their tiles
// fill the resident CTAs at least once, else blocks of 128 (4 rows per lane,
// four times as many tiles).  FP64: blocks of 128.
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
MsPlan ms_plan(const rbf_ctx* ctx, int64_t n, bool fp64) {
    static int occ[64] = {0};
    MsPlan pl{};
    const int64_t nb8 = (n + 255) / 256;
    const int64_t t8 = nb8 * (nb8 + 1) / 2;
    if (fp64) {
        pl.R = MD_R;
        pl.nb = (n + 32 * MD_R - 1) / (32 * MD_R);
    } else if (t8 >= (int64_t)ctx->sm_count *
                         pair_occupancy(occ, ctx, k_mf_sym<0, 8, double>, k_mf_sym<1, 8, double>, MS_W * 32, 4)) {
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
    return ms_plan(ctx, op->n, op->precision == RBF_FP64).G;
}

bool mf_slots_f32(const rbf_ctx* ctx, const rbf_operator* op) {
    return op->storage == RBF_MATRIX_FREE && op->precision != RBF_FP64 && ms_plan(ctx, op->n, false).k == 1;
}

int mf_part_rows(const rbf_ctx* ctx, const rbf_operator* op) {
    const MsPlan pl = ms_plan(ctx, op->n, op->precision == RBF_FP64);
    return (int)pl.nb + (pl.k > 1 ? pl.G : 0);
}

size_t mf_ws_bytes(const rbf_ctx* ctx, int64_t n) {
    int64_t rows = 0;
    for (bool fp64 : {false, true}) {
        const MsPlan pl = ms_plan(ctx, n, fp64);
        const int64_t r = pl.nb + (pl.k > 1 ? pl.G : 0);
        rows = r > rows ? r : rows;
    }
    return ws_align((size_t)rows * n * sizeof(double));
}

rbf_status launch_mf_partial(rbf_ctx* ctx, const rbf_operator* op, int trans, const double* x,
                             const float* x32, const float* X32, double* part, const int* done) {
    const double scale = op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0;
    const bool fp64 = op->precision == RBF_FP64;
    const MsPlan pl = ms_plan(ctx, op->n, fp64);
    if (pl.tiles > 2147483647LL) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large");
    const unsigned grid = (unsigned)pl.tiles;
    const int64_t n = op->n, ni = op->n_interior;
    double* slots = part + (pl.k > 1 ? (int64_t)pl.G * n : 0);  // folded: slots after the G group rows
    if (fp64) {
        if (!x) return rbf_fail(ctx, RBF_ERR_INTERNAL, "FP64 product without its input");
        const double c2 = op->c * op->c, k2 = op->k * op->k;
        if (trans) k_mf_sym_f64<1><<<grid, MS_W * 32, 0, ctx->stream>>>(op->d_nodes, n, ni, c2, k2, scale, x, pl.nb, slots, done);
        else k_mf_sym_f64<0><<<grid, MS_W * 32, 0, ctx->stream>>>(op->d_nodes, n, ni, c2, k2, scale, x, pl.nb, slots, done);
        RBF_LAUNCHED(ctx, "k_mf_sym_f64");
    } else {
        if (!X32 || !x32) return rbf_fail(ctx, RBF_ERR_INTERNAL, "FP32 product without its FP32 inputs");
        const float c2 = (float)(op->c * op->c), k2 = (float)(op->k * op->k);
#define MS_LAUNCH(T_, R_, S_) \
    k_mf_sym<T_, R_, S_><<<grid, MS_W * 32, 0, ctx->stream>>>(X32, n, ni, c2, k2, scale, x32, pl.nb, (S_*)slots, done)
        if (pl.k == 1) {  // FP32 slots
            if (pl.R == 8) {
                if (trans) MS_LAUNCH(1, 8, float);
                else MS_LAUNCH(0, 8, float);
            } else {
                if (trans) MS_LAUNCH(1, 4, float);
                else MS_LAUNCH(0, 4, float);
            }
        } else if (pl.R == 8) {
            if (trans) MS_LAUNCH(1, 8, double);
            else MS_LAUNCH(0, 8, double);
        } else {
            if (trans) MS_LAUNCH(1, 4, double);
            else MS_LAUNCH(0, 4, double);
        }
#undef MS_LAUNCH
        RBF_LAUNCHED(ctx, "k_mf_sym");
    }
    if (pl.k > 1) {
        k_ms_fold<<<dim3((unsigned)((n + 255) / 256), (unsigned)pl.G), 256, 0, ctx->stream>>>(part, n, (int)pl.nb, pl.k,
                                                                                             done);
        RBF_LAUNCHED(ctx, "k_ms_fold");
    }
    return RBF_OK;
}

RBF_CHECK_READER(mf)
