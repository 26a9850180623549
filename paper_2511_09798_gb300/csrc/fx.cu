// Exact fixed-point form of the FP64 assembled GKB products of Algorithm 1
// (r = A^T w, p = A z).
//
// GB300 executes FP64 FMAs at 2 per clock per SM (1.26 TFLOP/s).  An FP64
// matrix-vector product needs one FMA per 8-byte entry, so on this part the
// FP64 pipe, not HBM, bounds it (about 0.65 of the HBM copy rate).  These
// products take the FP64 pipe out of the inner loop:
//
// - once per GKB run A is copied into two 64-bit integer fixed-point forms,
//     NR_ij = round(A_ij 2^(1084 - ER_i))   (A z: rows share a scale),
//     NC_ij = round(A_ij 2^(1084 - EC_j))   (A^T w: columns share a scale),
//   ER_i / EC_j the largest biased exponent field in row i / column j, so
//   |N| < 2^62; entries within 2^-9 of their row's (column's) largest keep all
//   53 bits and every rounding error is at most 2^-62 of that largest entry;
// - each product rounds its vector the same way (scale from the vector's
//   largest exponent: the whole vector for A z, the CTA's row chunk for A^T w),
//   splits matrix and vector values into three 21-bit limbs and accumulates
//   the six limb products of weight >= 2^42 with 32 x 32 -> 64-bit integer
//   multiply-adds (mad.wide.s32).  The sums are exact.  The limb products left
//   out (weights 2^21 and 2^0) are below 2^-60 of the largest entry product
//   each, and since the vector's lower limbs are balanced (centred on zero)
//   they carry no bias;
// - each lane's three accumulators are rounded to FP64 once and then reduced
//   like the partial sums of the FP64 kernels.
//
// Error of an output (A^T w)_j: at most about 2^-61 (max_i |A_ij| sum_i |w_i|
// + sum_i |A_ij| max_i |w_i|) from the roundings to fixed point, plus the FP64
// roundings of the partials (likewise for A z by rows).  FP64 FMAs give
// n 2^-53 sum_i |A_ij w_i| at worst, ~sqrt(n) 2^-53 typically: when the
// entries of a row (column) and of the vector stay within about 2^8 of their
// largest, as in the collocation matrices, the fixed-point products are the
// more accurate; for rows or columns scaled over many orders of magnitude
// the bound above is normwise rather than componentwise.  The products read
// the same 8 bytes per entry as the FP64 ones and cost about ten integer
// instructions per entry instead of one FP64 FMA, which leaves HBM as the
// bound.  Non-finite entries set ER/EC = 2047 and a
// non-finite vector value sets its scale to 2047: the rows, columns or chunks
// concerned come out NaN, as in FP64 arithmetic, so the GKB breakdown test
// (code 3) sees them.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int FX_NONFINITE = 2047;
constexpr int FXN_THREADS = 512;  // A z: 16 warps, the vector's limbs in shared memory
constexpr int FXT_THREADS = 256;  // A^T w: 2 columns per thread, like the FP64 kernel
constexpr int FXT_UNROLL = 8;     // rows of loads in flight per thread (A^T w)
constexpr int FXE_THREADS = 256;  // exponent scan and conversion: 2 columns per thread

__device__ __forceinline__ int fx_exp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

__device__ __forceinline__ double fx_nan() { return __longlong_as_double(0x7FF8000000000000LL); }

// round(x 2^s) for |x| 2^s < 2^62 (s = 1084 - E with E at least the exponent
// field of x and at least 1); 0 for a non-finite x (flagged by E = 2047).
// Normal x: integer operations on the significand (the FP64 pipe is not used).
__device__ __forceinline__ long long fx_round(double x, int s) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) return 0;
    long long q;
    if (e == 0) {
        if ((b << 1) == 0) return 0;                // +-0
        q = __double2ll_rn(ldexp(fabs(x), s));      // subnormal: exact scaling, one rounding
    } else {
        const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;  // 53-bit significand
        const int d = 1075 - e - s;                 // |x| 2^s = m 2^-d with d >= -9
        if (d <= 0) q = m << (-d);
        else if (d > 54) q = 0;
        else q = (m + (1LL << (d - 1))) >> d;       // round half up
    }
    return b < 0 ? -q : q;
}

// Balanced 21-bit limbs of a vector value: q = z2 2^42 + z1 2^21 + z0 with
// z0, z1 in [-2^20, 2^20) and |z2| <= 2^20 + 1 (|q| < 2^62).
__device__ __forceinline__ int4 fx_limbs_bal(long long q) {
    const int z0 = (int)((q << 43) >> 43);
    q = (q - z0) >> 21;
    const int z1 = (int)((q << 43) >> 43);
    q = (q - z1) >> 21;
    return make_int4(z0, z1, (int)q, 0);
}

__device__ __forceinline__ long long imad_wide(int a, int b, long long c) {
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// acc += N * Z over the limb products of weight >= 2^42: N's limbs are its
// bit fields (a0, a1 in [0, 2^21), a2 = N >> 42 signed), Z's the balanced ones.
struct FxAcc {
    long long c2 = 0, c1 = 0, c0 = 0;  // weights 2^84, 2^63, 2^42
    __device__ __forceinline__ void add(long long N, int z0, int z1, int z2) {
        const unsigned lo = (unsigned)N, hi = (unsigned)(N >> 32);
        const int a0 = (int)(lo & 0x1FFFFFu);
        const int a1 = (int)(__funnelshift_r(lo, hi, 21) & 0x1FFFFFu);
        const int a2 = (int)hi >> 10;
        c2 = imad_wide(a2, z2, c2);
        c1 = imad_wide(a2, z1, c1);
        c1 = imad_wide(a1, z2, c1);
        c0 = imad_wide(a2, z0, c0);
        c0 = imad_wide(a1, z1, c0);
        c0 = imad_wide(a0, z2, c0);
    }
    // the accumulated value in units of 2^42, rounded to FP64
    __device__ __forceinline__ double value() const {
        return fma((double)c2, 0x1p42, fma((double)c1, 0x1p21, (double)c0));
    }
};

// value * 2^(e_mat + e_vec - 2126) (the units of FxAcc::value), NaN when
// either scale flags a non-finite value
__device__ __forceinline__ double fx_scale_out(double v, int e_mat, int e_vec) {
    if (e_mat == FX_NONFINITE || e_vec == FX_NONFINITE) return fx_nan();
    return ldexp(v, max(e_mat, 1) + max(e_vec, 1) - 2126);
}

// Largest exponent field of x[i0 .. i1) over the CTA (every thread gets it).
template <int NT>
__device__ __forceinline__ int fx_block_max_exp(const double* __restrict__ x, int64_t i0, int64_t i1, int* red) {
    int em = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += NT) em = max(em, fx_exp(__ldg(x + i)));
    em = __reduce_max_sync(RBF_FULL_MASK, em);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = em;
    __syncthreads();
    em = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) em = max(em, red[i]);
    return em;
}

// ---------------------------------------------------------------------------
// Row and column exponent tables: CTA (panel of 2 * FXE_THREADS columns, row
// chunk); the column maxima of the chunk and the row maxima of the panel are
// merged into rowE / colE (zeroed beforehand) with integer atomicMax.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(FXE_THREADS) k_fx_exps(const double* __restrict__ A, int64_t lda, int64_t n,
                                                         int chunks, int rows_max, int* __restrict__ rowE,
                                                         int* __restrict__ colE) {
    extern __shared__ int rmx[];  // [rows_max] row maxima of this panel
    const int q = blockIdx.x % chunks;
    const int pnl = blockIdx.x / chunks;
    const int64_t i0 = n * (int64_t)q / chunks;
    const int64_t i1 = n * (int64_t)(q + 1) / chunks;
    const int rows = (int)(i1 - i0);
    for (int r = threadIdx.x; r < rows; r += FXE_THREADS)
        if (RBF_IN_RANGE(r, rows_max)) rmx[r] = 0;
    __syncthreads();
    const int64_t c = (int64_t)pnl * (2 * FXE_THREADS) + 2 * threadIdx.x;
    const bool has0 = c < n, has1 = c + 1 < n;
    int cx = 0, cy = 0;
    for (int r = 0; r < rows; ++r) {
        int ex = 0, ey = 0;
        if (has0) {
            const double2 m = __ldcs(reinterpret_cast<const double2*>(A + (i0 + r) * lda + c));
            ex = fx_exp(m.x);
            ey = has1 ? fx_exp(m.y) : 0;
        }
        cx = max(cx, ex);
        cy = max(cy, ey);
        const int rm = __reduce_max_sync(RBF_FULL_MASK, max(ex, ey));
        if ((threadIdx.x & 31) == 0 && rm > 0 && RBF_IN_RANGE(r, rows_max)) atomicMax(&rmx[r], rm);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += FXE_THREADS)
        if (RBF_IN_RANGE(r, rows_max) && rmx[r] > 0) atomicMax(&rowE[i0 + r], rmx[r]);
    if (has0 && cx > 0) atomicMax(&colE[c], cx);
    if (has1 && cy > 0) atomicMax(&colE[c + 1], cy);
}

// NR and NC from A and the exponent tables (pad columns of an odd n: zero).
__global__ void __launch_bounds__(FXE_THREADS) k_fx_convert(const double* __restrict__ A, int64_t lda, int64_t n,
                                                            int chunks, const int* __restrict__ rowE,
                                                            const int* __restrict__ colE, long long* __restrict__ NR,
                                                            long long* __restrict__ NC) {
    const int q = blockIdx.x % chunks;
    const int pnl = blockIdx.x / chunks;
    const int64_t i0 = n * (int64_t)q / chunks;
    const int64_t i1 = n * (int64_t)(q + 1) / chunks;
    const int64_t c = (int64_t)pnl * (2 * FXE_THREADS) + 2 * threadIdx.x;
    if (c >= n) return;
    const bool has1 = c + 1 < n;
    const int scx = 1084 - max(colE[c], 1);
    const int scy = has1 ? 1084 - max(colE[c + 1], 1) : 0;
    for (int64_t i = i0; i < i1; ++i) {
        const double2 m = __ldcs(reinterpret_cast<const double2*>(A + i * lda + c));
        const int sr = 1084 - max(__ldg(rowE + i), 1);
        longlong2 r, k;
        r.x = fx_round(m.x, sr);
        k.x = fx_round(m.x, scx);
        r.y = has1 ? fx_round(m.y, sr) : 0;
        k.y = has1 ? fx_round(m.y, scy) : 0;
        *reinterpret_cast<longlong2*>(NR + i * lda + c) = r;
        *reinterpret_cast<longlong2*>(NC + i * lda + c) = k;
    }
}

// ---------------------------------------------------------------------------
// p = A z by the flat split (flat_bound) over W warps, on NR: every CTA first
// rounds the whole vector to fixed point at its largest exponent and keeps the
// balanced limbs in shared memory (three int arrays of stride nn, nn = n
// rounded up to even: 8-byte aligned int2 reads of column pairs).  Each row
// piece's lane sums are rounded once, reduced across the warp in FP64 and
// written to part[slot][row] as in the FP64 kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fx_pair(FxAcc& acc, const longlong2& m, const int* __restrict__ zs, int64_t nn,
                                        int64_t col) {
    const int2 z0 = *reinterpret_cast<const int2*>(zs + col);
    const int2 z1 = *reinterpret_cast<const int2*>(zs + nn + col);
    const int2 z2 = *reinterpret_cast<const int2*>(zs + 2 * nn + col);
    acc.add(m.x, z0.x, z1.x, z2.x);
    acc.add(m.y, z0.y, z1.y, z2.y);
}

__global__ void __launch_bounds__(FXN_THREADS) k_gemv_flat_fx(const long long* __restrict__ NR, int64_t ld,
                                                              int64_t n, const int* __restrict__ rowE,
                                                              const double* __restrict__ x, int64_t W, int chunks,
                                                              double* __restrict__ part, const int* __restrict__ done) {
    if (gkb_done(done)) return;
    extern __shared__ int zs[];  // [3][nn] limbs of x
    __shared__ int red[FXN_THREADS / 32];
    const int64_t nn = (n + 1) & ~(int64_t)1;
    const int ez = fx_block_max_exp<FXN_THREADS>(x, 0, n, red);
    const int sz = 1084 - max(ez, 1);
    for (int64_t j = threadIdx.x; j < n; j += FXN_THREADS) {
        const int4 l = fx_limbs_bal(fx_round(__ldg(x + j), sz));
        zs[j] = l.x;
        zs[nn + j] = l.y;
        zs[2 * nn + j] = l.z;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (FXN_THREADS / 32) + warp;
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
        const longlong2* __restrict__ row = reinterpret_cast<const longlong2*>(NR + r * ld + cs);
        const int* __restrict__ zc = zs + cs;
        const int64_t nvec = (ce - cs) >> 1;
        FxAcc acc;
        int64_t v = lane;
        for (; v + 224 < nvec; v += 256) {  // 8 loads of 16 bytes in flight per lane
            longlong2 m[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) m[u] = __ldcs(row + v + 32 * u);
#pragma unroll
            for (int u = 0; u < 8; ++u) fx_pair(acc, m[u], zc, nn, 2 * (v + 32 * u));
        }
        for (; v < nvec; v += 32) fx_pair(acc, __ldcs(row + v), zc, nn, 2 * v);
        if (((ce - cs) & 1) && lane == 0) {
            const int64_t col = ce - 1;
            acc.add(NR[r * ld + col], zs[col], zs[nn + col], zs[2 * nn + col]);
        }
        const double s = warp_sum(acc.value());
        if (lane == 0 && RBF_IN_RANGE(slot, chunks)) {
            part[(int64_t)slot * n + r] = fx_scale_out(s, __ldg(rowE + r), ez);
            if (ce == n)
                for (int s2 = slot + 1; s2 < chunks; ++s2) part[(int64_t)s2 * n + r] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// part[q][c] = sum over row chunk q of A_ic x_i, on NC: column panels x row
// chunks as the FP64 kernel; each CTA rounds its chunk of x at the chunk's own
// largest exponent (its partials are separate FP64 numbers, so the chunks need
// no common scale) and keeps the limbs (int4 per row, read as a broadcast) in
// shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(FXT_THREADS) k_gemv_t_fx(const long long* __restrict__ NC, int64_t ld, int64_t n,
                                                           const int* __restrict__ colE,
                                                           const double* __restrict__ x, int panel_cols, int chunks,
                                                           int rows_max, double* __restrict__ part,
                                                           const int* __restrict__ done) {
    if (gkb_done(done)) return;
    extern __shared__ int4 xl[];  // [rows_max] limbs of the chunk of x
    __shared__ int red[FXT_THREADS / 32];
    const int q = blockIdx.x % chunks;
    const int pnl = blockIdx.x / chunks;
    const int64_t i0 = n * (int64_t)q / chunks;
    int64_t i1 = n * (int64_t)(q + 1) / chunks;
    if (!RBF_IN_RANGE(i1 - i0, rows_max + 1)) i1 = i0 + rows_max;
    const int ex = fx_block_max_exp<FXT_THREADS>(x, i0, i1, red);
    const int sx = 1084 - max(ex, 1);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += FXT_THREADS) xl[i - i0] = fx_limbs_bal(fx_round(__ldg(x + i), sx));
    __syncthreads();
    const int64_t c = (int64_t)pnl * panel_cols + 2 * threadIdx.x;
    if (c >= n) return;
    const long long* __restrict__ base = NC + i0 * ld + c;
    FxAcc ax, ay;
    const int64_t rows = i1 - i0;
    int64_t r = 0;
    for (; r + FXT_UNROLL - 1 < rows; r += FXT_UNROLL) {
        longlong2 m[FXT_UNROLL];
#pragma unroll
        for (int u = 0; u < FXT_UNROLL; ++u) m[u] = __ldcs(reinterpret_cast<const longlong2*>(base + (r + u) * ld));
#pragma unroll
        for (int u = 0; u < FXT_UNROLL; ++u) {
            const int4 l = xl[r + u];
            ax.add(m[u].x, l.x, l.y, l.z);
            ay.add(m[u].y, l.x, l.y, l.z);
        }
    }
    for (; r < rows; ++r) {
        const longlong2 m = __ldcs(reinterpret_cast<const longlong2*>(base + r * ld));
        const int4 l = xl[r];
        ax.add(m.x, l.x, l.y, l.z);
        ay.add(m.y, l.x, l.y, l.z);
    }
    part[(int64_t)q * n + c] = fx_scale_out(ax.value(), __ldg(colE + c), ex);
    if (c + 1 < n) part[(int64_t)q * n + c + 1] = fx_scale_out(ay.value(), __ldg(colE + c + 1), ex);
}

constexpr int64_t FX_MAX_N = 16384;  // the vector's limbs of A z fit in shared memory (196 KB)

size_t fxn_smem(int64_t n) { return (size_t)3 * ((n + 1) & ~(int64_t)1) * sizeof(int); }

// CTAs of k_gemv_flat_fx resident per SM at this n (cached per device for the
// last n asked; the shared-memory limit is raised once to the largest size).
// Contexts on different host threads share the cache, hence the mutex.
int fxn_per_sm(const rbf_ctx* ctx, int64_t n) {
    static std::mutex mu;
    static int64_t last_n[64] = {0};
    static int last_per[64] = {0};
    static bool raised[64] = {false};
    std::lock_guard<std::mutex> lock(mu);
    const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
    if (last_n[dev] == n && last_per[dev] > 0) return last_per[dev];
    if (!raised[dev]) {
        if (cudaFuncSetAttribute((const void*)k_gemv_flat_fx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fxn_smem(FX_MAX_N)) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        raised[dev] = true;
    }
    int a = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_gemv_flat_fx, FXN_THREADS, fxn_smem(n)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    last_n[dev] = n;
    last_per[dev] = a;
    return a;
}

void fxn_plan(const rbf_ctx* ctx, int64_t n, int* grid, int64_t* W, int* chunks) {
    int per = fxn_per_sm(ctx, n);
    if (per < 1) per = 1;
    flat_split_plan(n, (int64_t)ctx->sm_count * per * (FXN_THREADS / 32), W, chunks);
    *grid = (int)((*W + FXN_THREADS / 32 - 1) / (FXN_THREADS / 32));
}

// A^T w plan (the FP64 kernel's panels and chunks) and its largest chunk.
void fxt_plan(const rbf_ctx* ctx, int64_t n, int* panel_cols, int* panels, int* chunks, int* rows_max) {
    plan_t(ctx, n, 2, panel_cols, panels, chunks);
    int64_t rm = 0;
    for (int q = 0; q < *chunks; ++q) {
        const int64_t r = n * (int64_t)(q + 1) / *chunks - n * (int64_t)q / *chunks;
        if (r > rm) rm = r;
    }
    *rows_max = (int)rm;
}

}  // namespace

bool fx_eligible(const rbf_ctx* ctx, const rbf_operator* op) {
    return op->storage == RBF_ASSEMBLED && op->precision == RBF_FP64 && !ctx->opt.fma_products && op->n >= 1 &&
           op->n <= FX_MAX_N;
}

size_t fx_ws_bytes(const rbf_operator* op) {
    return 2 * ws_align((size_t)op->n * (size_t)op->lda * sizeof(long long)) +
           2 * ws_align((size_t)op->n * sizeof(int));
}

FxCopies fx_carve(WsCarve& wc, const rbf_operator* op) {
    FxCopies f;
    f.NR = wc.take<long long>((size_t)op->n * (size_t)op->lda);
    f.NC = wc.take<long long>((size_t)op->n * (size_t)op->lda);
    f.rowE = wc.take<int>((size_t)op->n);
    f.colE = wc.take<int>((size_t)op->n);
    return f;
}

int fx_n_chunks(const rbf_ctx* ctx, int64_t n) {
    int g, ch;
    int64_t W;
    fxn_plan(ctx, n, &g, &W, &ch);
    return ch;
}

rbf_status launch_fx_prepare(rbf_ctx* ctx, const rbf_operator* op, const FxCopies& f) {
    const int64_t n = op->n;
    int pc, pn, ch, rows_max;
    fxt_plan(ctx, n, &pc, &pn, &ch, &rows_max);
    // the exponent scan and the conversion cover 2 * FXE_THREADS columns per panel
    if (pc != 2 * FXE_THREADS)
        return rbf_fail(ctx, RBF_ERR_INTERNAL, "fixed-point copies: panel of %d columns, kernels cover %d", pc,
                        2 * FXE_THREADS);
    RBF_CUDA(ctx, cudaMemsetAsync(f.rowE, 0, (size_t)n * sizeof(int), ctx->stream));
    RBF_CUDA(ctx, cudaMemsetAsync(f.colE, 0, (size_t)n * sizeof(int), ctx->stream));
    const size_t smem = (size_t)rows_max * sizeof(int);
    if (smem > 48 * 1024)
        RBF_CUDA(ctx, cudaFuncSetAttribute((const void*)k_fx_exps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    k_fx_exps<<<pn * ch, FXE_THREADS, smem, ctx->stream>>>((const double*)op->d_A, op->lda, n, ch, rows_max,
                                                           f.rowE, f.colE);
    RBF_LAUNCHED(ctx, "k_fx_exps");
    k_fx_convert<<<pn * ch, FXE_THREADS, 0, ctx->stream>>>((const double*)op->d_A, op->lda, n, ch, f.rowE, f.colE,
                                                          f.NR, f.NC);
    RBF_LAUNCHED(ctx, "k_fx_convert");
    return RBF_OK;
}

rbf_status launch_fx_n(rbf_ctx* ctx, const rbf_operator* op, const FxCopies& f, const double* x, double* part,
                       const int* done) {
    int g, ch;
    int64_t W;
    fxn_plan(ctx, op->n, &g, &W, &ch);
    k_gemv_flat_fx<<<g, FXN_THREADS, fxn_smem(op->n), ctx->stream>>>(f.NR, op->lda, op->n, f.rowE, x, W, ch, part,
                                                                      done);
    RBF_LAUNCHED(ctx, "k_gemv_flat_fx");
    return RBF_OK;
}

rbf_status launch_fx_t(rbf_ctx* ctx, const rbf_operator* op, const FxCopies& f, const double* x, double* part,
                       const int* done) {
    int pc, pn, ch, rows_max;
    fxt_plan(ctx, op->n, &pc, &pn, &ch, &rows_max);
    const size_t smem = (size_t)rows_max * sizeof(int4);
    if (smem > 48 * 1024)
        RBF_CUDA(ctx, cudaFuncSetAttribute((const void*)k_gemv_t_fx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    k_gemv_t_fx<<<pn * ch, FXT_THREADS, smem, ctx->stream>>>(f.NC, op->lda, op->n, f.colE, x, pc, ch, rows_max,
                                                            part, done);
    RBF_LAUNCHED(ctx, "k_gemv_t_fx");
    return RBF_OK;
}

RBF_CHECK_READER(fx)
