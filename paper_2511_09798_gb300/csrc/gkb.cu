// Golub-Kahan bidiagonalization with full reorthogonalization (Algorithm 1).
//
// One half-step (r-side: r = A^T w_j - beta_j z_{j-1}; p-side: p = A z_j -
// alpha_j w_j) is a fixed chain of kernels on the context stream:
//
//   finalize  1 CTA   nrm = |q_raw| from per-slab partials; breakdown test
//                     (tau = factor * N * eps * c_hat); stores alpha_j or beta_j
//   product           partial sums of A^T q_raw or A q_raw (assembled or
//                     matrix-free), one row of partials per chunk
//   R1        slab    v = (sum of partials) / nrm - nrm * u;  writes the
//                     normalised previous vector q_raw / nrm into its basis;
//                     per-slab partials of Q^T v
//   reduce            h = Q^T v
//   R2        slab    v -= Q h; per-slab partials of Q^T v
//   reduce            h = Q^T v
//   R3        slab    v -= Q h; per-slab partials of |v|^2 (+ FP32 copy of v)
//
// i.e. classical Gram-Schmidt applied twice ("twice is enough") against the
// current basis before the norm, which is the reorthogonalization placement
// chosen for Algorithm 1 step 7.  All reductions are deterministic (fixed
// order), so repeated runs are bitwise identical.  Once a breakdown is found the
// finalize kernel sets a device flag and every later kernel of the run returns
// immediately.
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int SL_THREADS = 256;
constexpr int SL_WARPS = SL_THREADS / 32;
constexpr int SL_MAX_ROWS = 2048;  // slab rows held in shared memory
constexpr int UPD_ROWS = 64;       // rows per update pass
constexpr int UPD_GROUPS = SL_THREADS / UPD_ROWS;

struct Slab {
    int64_t r0, r1;
};
__device__ __forceinline__ Slab slab_of(int64_t n) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    Slab s;
    s.r0 = (int64_t)blockIdx.x * per;
    s.r1 = min(n, s.r0 + per);
    if (s.r1 < s.r0) s.r1 = s.r0;
    return s;
}

// hpart[m * G + b] = sum_{i in slab b} Q[m][i] v[i]   (warp per basis vector)
__device__ __forceinline__ void slab_dot(const double* __restrict__ Q, int64_t ldq, int mcount,
                                         const double* __restrict__ vs, Slab s,
                                         double* __restrict__ hpart) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rows = s.r1 - s.r0;
    for (int m = warp; m < mcount; m += SL_WARPS) {
        const double* __restrict__ q = Q + (int64_t)m * ldq + s.r0;
        double acc = 0.0;
        for (int64_t i = lane; i < rows; i += 32) acc = fma(q[i], vs[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) hpart[(int64_t)m * gridDim.x + blockIdx.x] = acc;
    }
}

// vs[i] -= sum_m Q[m][i] h[m] for the slab rows.
__device__ __forceinline__ void slab_update(const double* __restrict__ Q, int64_t ldq, int mcount,
                                            const double* __restrict__ hs, double* __restrict__ vs,
                                            Slab s, double* red /* [UPD_GROUPS][UPD_ROWS] */) {
    const int row = threadIdx.x % UPD_ROWS;
    const int grp = threadIdx.x / UPD_ROWS;
    const int64_t rows = s.r1 - s.r0;
    for (int64_t base = 0; base < rows; base += UPD_ROWS) {
        const int64_t i = base + row;
        double acc = 0.0;
        if (i < rows) {
            const double* __restrict__ q = Q + s.r0 + i;
            for (int m = grp; m < mcount; m += UPD_GROUPS) acc = fma(q[(int64_t)m * ldq], hs[m], acc);
        }
        red[grp * UPD_ROWS + row] = acc;
        __syncthreads();
        if (grp == 0 && i < rows) {
            double t = 0.0;
#pragma unroll
            for (int g = 0; g < UPD_GROUPS; ++g) t += red[g * UPD_ROWS + row];
            vs[i] -= t;
        }
        __syncthreads();
    }
}

// Block-wide deterministic sum of v over [0, count).
__device__ double block_sum(const double* __restrict__ v, int64_t count, double* red) {
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc += v[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// finalize: nrm = sqrt(sum npart).  side 0 = beta (r-side start / final),
// side 1 = alpha (p-side start).  j is the 1-based step.
// ---------------------------------------------------------------------------
__global__ void k_finalize(rbf_dev_state* __restrict__ stt, const double* __restrict__ npart, int G,
                           int side, int j, int64_t n, double factor, double* __restrict__ alpha,
                           double* __restrict__ beta, double* __restrict__ wzero /* W col j or null */,
                           int final_step) {
    __shared__ double red[32];
    __shared__ int bd;
    if (stt->info[IN_DONE]) return;
    double s = block_sum(npart, G, red);
    if (threadIdx.x == 0) {
        double nrm = sqrt(s);
        double* sc = stt->scal;
        const double eps = DBL_EPSILON;
        int brk = 0;
        if (side == 1) {  // alpha_j
            double tau = factor * (double)n * eps * fmax(sc[SC_CHAT0], nrm);
            if (nrm <= tau) {
                brk = 1;
                stt->info[IN_STEPS] = j - 1;
                stt->info[IN_BREAK] = 1;
                stt->info[IN_DONE] = 1;
            } else {
                alpha[j - 1] = nrm;
                sc[SC_ALPHA] = nrm;
                sc[SC_INV_ALPHA] = 1.0 / nrm;
            }
        } else if (j == 1) {  // beta_1 = |f|
            if (!(nrm > 0.0)) {
                brk = 1;
                stt->info[IN_STEPS] = 0;
                stt->info[IN_BREAK] = 1;
                stt->info[IN_DONE] = 1;
            } else {
                beta[0] = nrm;
                sc[SC_BETA] = nrm;
                sc[SC_INV_BETA] = 1.0 / nrm;
                sc[SC_CHAT0] = 0.0;
            }
        } else {  // beta_j closes step j-1
            double ch = fmax(sc[SC_CHAT0], hypot(alpha[j - 2], nrm));
            sc[SC_CHAT0] = ch;
            double tau = factor * (double)n * eps * ch;
            if (nrm <= tau) {
                brk = 2;
                beta[j - 1] = 0.0;
                stt->info[IN_STEPS] = j - 1;
                stt->info[IN_BREAK] = 2;
                stt->info[IN_DONE] = 1;
            } else {
                beta[j - 1] = nrm;
                sc[SC_BETA] = nrm;
                sc[SC_INV_BETA] = 1.0 / nrm;
                stt->info[IN_STEPS] = j - 1;
                if (final_step) stt->info[IN_DONE] = 1;
            }
        }
        bd = brk;
    }
    __syncthreads();
    if (bd == 2 && wzero)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) wzero[i] = 0.0;
}

// ---------------------------------------------------------------------------
// R1: v = inv * sum_q part[q][i] - nrm * u[i]; basis_out = q_raw * inv;
//     hpart = Q^T v (mcount vectors)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SL_THREADS) k_r1(const rbf_dev_state* __restrict__ stt, int64_t n,
                                                   int chunks, const double* __restrict__ part,
                                                   int inv_idx, int nrm_idx,
                                                   const double* __restrict__ u,
                                                   const double* __restrict__ q_raw,
                                                   double* __restrict__ basis_out,
                                                   double* __restrict__ v_out,
                                                   const double* __restrict__ Q, int64_t ldq,
                                                   int mcount, double* __restrict__ hpart) {
    if (stt->info[IN_DONE]) return;
    __shared__ double vs[SL_MAX_ROWS];
    const Slab s = slab_of(n);
    const double inv = stt->scal[inv_idx];
    const double nrm = stt->scal[nrm_idx];
    for (int64_t i = s.r0 + threadIdx.x; i < s.r1; i += SL_THREADS) {
        double acc = 0.0;
        for (int q = 0; q < chunks; ++q) acc += part[(int64_t)q * n + i];
        double v = acc * inv;
        if (u) v = fma(-nrm, u[i], v);
        v_out[i] = v;
        vs[i - s.r0] = v;
        if (basis_out) basis_out[i] = q_raw[i] * inv;
    }
    __syncthreads();
    slab_dot(Q, ldq, mcount, vs, s, hpart);
}

// h[m] = sum_b hpart[m * G + b]   (warp per m)
__global__ void k_reduce_h(const rbf_dev_state* __restrict__ stt, const double* __restrict__ hpart,
                           int G, int mcount, double* __restrict__ h) {
    if (stt->info[IN_DONE]) return;
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= mcount) return;
    double acc = 0.0;
    for (int b = lane; b < G; b += 32) acc += hpart[(int64_t)m * G + b];
    acc = warp_sum(acc);
    if (lane == 0) h[m] = acc;
}

// R2 (mode 0): v -= Q h; hpart = Q^T v.   R3 (mode 1): v -= Q h; npart = |v|^2 (+ v32).
__global__ void __launch_bounds__(SL_THREADS) k_r23(const rbf_dev_state* __restrict__ stt, int64_t n,
                                                    double* __restrict__ v,
                                                    const double* __restrict__ Q, int64_t ldq,
                                                    int mcount, const double* __restrict__ h,
                                                    int mode, double* __restrict__ hpart,
                                                    double* __restrict__ npart,
                                                    float* __restrict__ v32) {
    if (stt->info[IN_DONE]) return;
    __shared__ double vs[SL_MAX_ROWS];
    __shared__ double hs[1024];
    __shared__ double red[UPD_GROUPS * UPD_ROWS];
    const Slab s = slab_of(n);
    const int64_t rows = s.r1 - s.r0;
    for (int m = threadIdx.x; m < mcount; m += SL_THREADS) hs[m] = h[m];
    for (int64_t i = threadIdx.x; i < rows; i += SL_THREADS) vs[i] = v[s.r0 + i];
    __syncthreads();
    if (mcount > 0) slab_update(Q, ldq, mcount, hs, vs, s, red);
    for (int64_t i = threadIdx.x; i < rows; i += SL_THREADS) {
        v[s.r0 + i] = vs[i];
        if (mode == 1 && v32) v32[s.r0 + i] = (float)vs[i];
    }
    __syncthreads();
    if (mode == 0) {
        slab_dot(Q, ldq, mcount, vs, s, hpart);
    } else {
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < rows; i += SL_THREADS) acc = fma(vs[i], vs[i], acc);
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < SL_WARPS; ++w) t += red[w];
            npart[blockIdx.x] = t;
        }
    }
}

// Squared norm partials of an input vector (start of the run) + FP32 copy.
__global__ void __launch_bounds__(SL_THREADS) k_norm_partials(int64_t n, const double* __restrict__ x,
                                                              double* __restrict__ npart,
                                                              double* __restrict__ copy,
                                                              float* __restrict__ x32) {
    __shared__ double red[SL_WARPS];
    const Slab s = slab_of(n);
    double acc = 0.0;
    for (int64_t i = s.r0 + threadIdx.x; i < s.r1; i += SL_THREADS) {
        double t = x[i];
        acc = fma(t, t, acc);
        if (copy) copy[i] = t;
        if (x32) x32[i] = (float)t;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < SL_WARPS; ++w) t += red[w];
        npart[blockIdx.x] = t;
    }
}

// basis_out = q_raw * scal[inv_idx] (the last w_{l+1}).
__global__ void k_write_basis(const rbf_dev_state* __restrict__ stt, int64_t n, int inv_idx,
                              const double* __restrict__ q_raw, double* __restrict__ out) {
    if (stt->info[IN_BREAK] != 0) return;
    const double inv = stt->scal[inv_idx];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = q_raw[i] * inv;
}

__global__ void k_reset_state(rbf_dev_state* stt, int steps_done, double beta_now, double c_hat,
                              int resume) {
    if (threadIdx.x == 0) {
        for (int t = 0; t < 8; ++t) stt->info[t] = 0;
        stt->info[IN_STEPS] = steps_done;
        stt->scal[SC_CHAT0] = c_hat;
        if (resume) {
            stt->scal[SC_BETA] = beta_now;
            stt->scal[SC_INV_BETA] = 1.0;  // q_raw is the stored, already normalised w
        }
    }
}

}  // namespace

static int slab_grid(const rbf_ctx* ctx, int64_t n) {
    int64_t g = ctx->sm_count;
    int64_t need = (n + SL_MAX_ROWS - 1) / SL_MAX_ROWS;
    if (g < need) g = need;
    if (g > n) g = n;
    return (int)(g < 1 ? 1 : g);
}

static int product_chunks(const rbf_ctx* ctx, const rbf_operator* op, int trans) {
    if (op->storage == RBF_MATRIX_FREE) return mf_chunks(ctx, op);
    return trans ? gemv_t_chunks(ctx, op) : 1;
}

size_t gkb_ws_bytes(const rbf_ctx* ctx, int64_t n, int steps, int precision) {
    (void)precision;
    rbf_operator fake{};
    fake.n = n;
    fake.precision = RBF_MIXED;
    fake.storage = RBF_MATRIX_FREE;
    int ch = mf_chunks(ctx, &fake);
    fake.storage = RBF_ASSEMBLED;
    int ch2 = gemv_t_chunks(ctx, &fake);
    fake.precision = RBF_FP64;
    int ch3 = gemv_t_chunks(ctx, &fake);
    if (ch2 > ch) ch = ch2;
    if (ch3 > ch) ch = ch3;
    const int G = slab_grid(ctx, n);
    size_t b = 0;
    b += ws_align((size_t)ch * n * 8);                // partials
    b += 2 * ws_align((size_t)n * 8);                 // vr, vp
    b += 2 * ws_align((size_t)n * 4);                 // vr32, vp32
    b += ws_align((size_t)(steps + 2) * G * 8);       // hpart
    b += ws_align((size_t)(steps + 2) * 8);           // h
    b += ws_align((size_t)G * 8);                     // npart
    return b + 4096;
}

// Launch the product "part = M q_raw" for one half-step.
static rbf_status gkb_product(rbf_ctx* ctx, const rbf_operator* op, int trans, const double* q_raw,
                              const float* q32, double* part, const int* done) {
    const int slot = rbf_prod_begin(ctx, trans);
    rbf_status st;
    if (op->storage == RBF_MATRIX_FREE) st = launch_mf_partial(ctx, op, trans, q32, part, done);
    else if (trans) st = launch_gemv_t_partial(ctx, op, q_raw, q32, part, done);
    else st = launch_gemv_n(ctx, op, q_raw, q32, part, nullptr, nullptr, nullptr, done);
    rbf_prod_end(ctx, trans, slot);
    return st;
}

rbf_status gkb_run(rbf_ctx* ctx, const rbf_operator* op, const double* f, int j_begin, int j_end,
                   rbf_gkb_state* st) {
    const int64_t n = op->n;
    const int G = slab_grid(ctx, n);
    if ((n + G - 1) / G > SL_MAX_ROWS) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large for slab kernels");
    if (st->capacity + 1 > 1024) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "capacity above 1023 steps");
    RBF_TRY(rbf_ws_reserve(ctx, gkb_ws_bytes(ctx, n, st->capacity, op->precision)));
    WsCarve wc(ctx->ws);
    const int chT = product_chunks(ctx, op, 1), chN = product_chunks(ctx, op, 0);
    double* part = wc.take<double>((size_t)(chT > chN ? chT : chN) * n);
    double* vr = wc.take<double>((size_t)n);
    double* vp = wc.take<double>((size_t)n);
    float* vr32 = wc.take<float>((size_t)n);
    float* vp32 = wc.take<float>((size_t)n);
    double* hpart = wc.take<double>((size_t)(st->capacity + 2) * G);
    double* h = wc.take<double>((size_t)(st->capacity + 2));
    double* npart = wc.take<double>((size_t)G);
    rbf_dev_state* dst = ctx->d_state;
    const int* done = &dst->info[IN_DONE];
    const bool mixed = op->precision == RBF_MIXED;
    const double factor = ctx->opt.breakdown_factor;
    cudaStream_t s = ctx->stream;
    double* W = st->d_W;
    double* Z = st->d_Z;
    const int64_t ldw = st->ldw, ldz = st->ldz;

    // q_raw for the first r-side: f (fresh run) or the stored w_{j_begin} (resume)
    const double* q_raw = vp;
    if (j_begin == 1) {
        k_reset_state<<<1, 32, 0, s>>>(dst, 0, 0.0, 0.0, 0);
        RBF_LAUNCHED(ctx, "k_reset_state");
        k_norm_partials<<<G, SL_THREADS, 0, s>>>(n, f, npart, vp, mixed ? vp32 : nullptr);
        RBF_LAUNCHED(ctx, "k_norm_partials");
    } else {
        // resume: beta_{j_begin} and w_{j_begin} are stored in the state
        double beta_now = 0.0;
        RBF_CUDA(ctx, cudaMemcpyAsync(&beta_now, st->d_beta + (j_begin - 1), sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
        RBF_CUDA(ctx, cudaStreamSynchronize(s));
        k_reset_state<<<1, 32, 0, s>>>(dst, j_begin - 1, beta_now, st->c_hat, 1);
        RBF_LAUNCHED(ctx, "k_reset_state");
        q_raw = W + (int64_t)(j_begin - 1) * ldw;
        k_norm_partials<<<G, SL_THREADS, 0, s>>>(n, q_raw, npart, vp, mixed ? vp32 : nullptr);
        RBF_LAUNCHED(ctx, "k_norm_partials");
        q_raw = vp;
    }
    const unsigned red_grid = (unsigned)((st->capacity + 2 + 7) / 8);
    for (int j = j_begin; j <= j_end; ++j) {
        // ---------------- r-side: r = A^T w_j - beta_j z_{j-1} ----------------
        if (!(j == j_begin && j_begin > 1)) {
            k_finalize<<<1, 256, 0, s>>>(dst, npart, G, 0, j, n, factor, st->d_alpha, st->d_beta,
                                         W + (int64_t)(j - 1) * ldw, 0);
            RBF_LAUNCHED(ctx, "k_finalize");
        }
        RBF_TRY(gkb_product(ctx, op, 1, q_raw, vp32, part, done));
        const int mz = j - 1;
        k_r1<<<G, SL_THREADS, 0, s>>>(dst, n, chT, part, SC_INV_BETA, SC_BETA,
                                      j >= 2 ? Z + (int64_t)(j - 2) * ldz : nullptr, q_raw,
                                      W + (int64_t)(j - 1) * ldw, vr, Z, ldz, mz, hpart);
        RBF_LAUNCHED(ctx, "k_r1");
        k_reduce_h<<<red_grid, 256, 0, s>>>(dst, hpart, G, mz, h);
        RBF_LAUNCHED(ctx, "k_reduce_h");
        k_r23<<<G, SL_THREADS, 0, s>>>(dst, n, vr, Z, ldz, mz, h, 0, hpart, npart, nullptr);
        RBF_LAUNCHED(ctx, "k_r23");
        k_reduce_h<<<red_grid, 256, 0, s>>>(dst, hpart, G, mz, h);
        RBF_LAUNCHED(ctx, "k_reduce_h");
        k_r23<<<G, SL_THREADS, 0, s>>>(dst, n, vr, Z, ldz, mz, h, 1, hpart, npart,
                                       mixed ? vr32 : nullptr);
        RBF_LAUNCHED(ctx, "k_r23");
        // ---------------- p-side: p = A z_j - alpha_j w_j ----------------
        k_finalize<<<1, 256, 0, s>>>(dst, npart, G, 1, j, n, factor, st->d_alpha, st->d_beta,
                                     nullptr, 0);
        RBF_LAUNCHED(ctx, "k_finalize");
        RBF_TRY(gkb_product(ctx, op, 0, vr, vr32, part, done));
        const int mw = j;
        k_r1<<<G, SL_THREADS, 0, s>>>(dst, n, chN, part, SC_INV_ALPHA, SC_ALPHA,
                                      W + (int64_t)(j - 1) * ldw, vr, Z + (int64_t)(j - 1) * ldz, vp,
                                      W, ldw, mw, hpart);
        RBF_LAUNCHED(ctx, "k_r1");
        k_reduce_h<<<red_grid, 256, 0, s>>>(dst, hpart, G, mw, h);
        RBF_LAUNCHED(ctx, "k_reduce_h");
        k_r23<<<G, SL_THREADS, 0, s>>>(dst, n, vp, W, ldw, mw, h, 0, hpart, npart, nullptr);
        RBF_LAUNCHED(ctx, "k_r23");
        k_reduce_h<<<red_grid, 256, 0, s>>>(dst, hpart, G, mw, h);
        RBF_LAUNCHED(ctx, "k_reduce_h");
        k_r23<<<G, SL_THREADS, 0, s>>>(dst, n, vp, W, ldw, mw, h, 1, hpart, npart,
                                       mixed ? vp32 : nullptr);
        RBF_LAUNCHED(ctx, "k_r23");
        q_raw = vp;
    }
    // beta_{l+1} and w_{l+1}
    k_finalize<<<1, 256, 0, s>>>(dst, npart, G, 0, j_end + 1, n, factor, st->d_alpha, st->d_beta,
                                 W + (int64_t)j_end * ldw, 1);
    RBF_LAUNCHED(ctx, "k_finalize");
    k_write_basis<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dst, n, SC_INV_BETA, vp,
                                                              W + (int64_t)j_end * ldw);
    RBF_LAUNCHED(ctx, "k_write_basis");
    return RBF_OK;
}

static rbf_status check_state(rbf_ctx* ctx, const rbf_operator* op, const rbf_gkb_state* st, int steps) {
    if (!op) return rbf_fail(ctx, RBF_ERR_INVALID, "op is NULL");
    if (!st || !st->d_W || !st->d_Z || !st->d_alpha || !st->d_beta)
        return rbf_fail(ctx, RBF_ERR_INVALID, "GKB state buffers missing");
    if (st->n != op->n) return rbf_fail(ctx, RBF_ERR_INVALID, "state n differs from operator n");
    if (st->ldw < op->n || st->ldz < op->n) return rbf_fail(ctx, RBF_ERR_INVALID, "ldw/ldz < n");
    if (steps < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "steps must be >= 1");
    if (steps > st->capacity) return rbf_fail(ctx, RBF_ERR_INVALID, "steps exceed the state capacity");
    if (steps > op->n) return rbf_fail(ctx, RBF_ERR_INVALID, "steps exceed n");
    if (op->storage == RBF_ASSEMBLED && !op->d_A) return rbf_fail(ctx, RBF_ERR_INVALID, "no matrix");
    return RBF_OK;
}

static rbf_status read_back(rbf_ctx* ctx, rbf_gkb_state* st) {
    RBF_CUDA(ctx, cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(rbf_dev_state),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RBF_CUDA(ctx, cudaGetLastError());
    st->steps_done = ctx->h_state->info[IN_STEPS];
    st->breakdown = ctx->h_state->info[IN_BREAK];
    st->c_hat = ctx->h_state->scal[SC_CHAT0];
    return RBF_OK;
}

extern "C" rbf_status rbf_gkb(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int steps,
                              rbf_gkb_state* st) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!d_f) return rbf_fail(ctx, RBF_ERR_INVALID, "d_f is NULL");
    RBF_TRY(check_state(ctx, op, st, steps));
    rbf_timer_start(ctx);
    RBF_TRY(gkb_run(ctx, op, d_f, 1, steps, st));
    RBF_TRY(read_back(ctx, st));
    ctx->tim.gkb_ms = rbf_timer_stop(ctx);
    ctx->tim.gkb_steps = st->steps_done;
    return RBF_OK;
}

extern "C" rbf_status rbf_gkb_resume(rbf_ctx* ctx, const rbf_operator* op, rbf_gkb_state* st,
                                     int more_steps) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!st) return rbf_fail(ctx, RBF_ERR_INVALID, "state is NULL");
    if (st->breakdown != 0 || more_steps == 0) return RBF_OK;
    const int l0 = st->steps_done;
    if (l0 < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "resume needs a state with steps_done >= 1");
    RBF_TRY(check_state(ctx, op, st, l0 + more_steps));
    rbf_timer_start(ctx);
    RBF_TRY(gkb_run(ctx, op, nullptr, l0 + 1, l0 + more_steps, st));
    RBF_TRY(read_back(ctx, st));
    ctx->tim.gkb_ms = rbf_timer_stop(ctx);
    ctx->tim.gkb_steps = st->steps_done - l0;
    return RBF_OK;
}
