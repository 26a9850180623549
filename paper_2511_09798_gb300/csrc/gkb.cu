// Golub-Kahan bidiagonalization with full reorthogonalization (Algorithm 1).
//
// One half-step (r-side: r = A^T w_j - beta_j z_{j-1}; p-side: p = A z_j -
// alpha_j w_j) is two launches on the context stream:
//
//   product   partial sums of A^T q_raw or A q_raw (assembled or matrix-free),
//             one row of partials per chunk (q_raw unnormalised)
//   k_half    one cooperative kernel, one CTA per SM, each CTA owning a slab
//             of rows:  finalize nrm = |q_raw| from the previous |v|^2
//             partials (alpha_j or beta_j, breakdown test tau = factor * N *
//             eps * c_hat) -> v = (sum of partials) / nrm - nrm * u, store
//             q_raw / nrm into its basis -> [per-slab Q^T v partials, one
//             grid barrier that also sums them into h, v -= Q h] twice
//             -> |v|^2 partials.  The CTA's slabs of Q, u, q_raw and the
//             product partials are staged in shared memory (cp.async).
//
// i.e. classical Gram-Schmidt applied twice ("twice is enough") against the
// current basis before the norm, which is the reorthogonalization placement
// chosen for Algorithm 1 step 7.  All reductions are deterministic (fixed
// order), so repeated runs are bitwise identical.  Grid barriers poll a bounded
// number of times and report RBF_ERR_TIMEOUT instead of hanging.  Once a
// breakdown is found a device flag makes every later kernel return at once.
#include <algorithm>
#include <cfloat>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "grid_sync.cuh"

namespace {

constexpr int SL_THREADS = 256;
constexpr int SL_WARPS = SL_THREADS / 32;
constexpr int SL_MAX_ROWS = 2048;  // slab rows held in shared memory
constexpr int UPD_ROWS = 64;       // rows per update pass
constexpr int UPD_GROUPS = SL_THREADS / UPD_ROWS;
constexpr int SPLIT = 4;           // threads per row (partial sums) and per basis vector (dots)

struct Slab {
    int64_t r0, r1;
};
// Balanced contiguous partition: CTA b owns rows [n b / G, n (b+1) / G).
__device__ __forceinline__ Slab slab_of(int64_t n) {
    Slab s;
    s.r0 = n * (int64_t)blockIdx.x / gridDim.x;
    s.r1 = n * (int64_t)(blockIdx.x + 1) / gridDim.x;
    return s;
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
            const bool nonfinite = !isfinite(nrm);
            if (nrm <= tau || nonfinite) {
                brk = 1;
                stt->info[IN_STEPS] = j - 1;
                stt->info[IN_BREAK] = nonfinite ? 3 : 1;
                stt->info[IN_DONE] = 1;
            } else {
                alpha[j - 1] = nrm;
                sc[SC_ALPHA] = nrm;
                sc[SC_INV_ALPHA] = 1.0 / nrm;
            }
        } else if (j == 1) {  // beta_1 = |f|
            const bool nonfinite = !isfinite(nrm);
            if (!(nrm > 0.0) || nonfinite) {
                brk = 1;
                stt->info[IN_STEPS] = 0;
                stt->info[IN_BREAK] = nonfinite ? 3 : 1;
                stt->info[IN_DONE] = 1;
            } else {
                beta[0] = nrm;
                sc[SC_BETA] = nrm;
                sc[SC_INV_BETA] = 1.0 / nrm;
                sc[SC_CHAT0] = 0.0;
            }
        } else {  // beta_j closes step j-1 (c_hat slot j&1 in, both slots out)
            double ch = fmax(sc[SC_CHAT0 + (j & 1)], hypot(alpha[j - 2], nrm));
            const bool nonfinite = !isfinite(nrm);
            if (!nonfinite) {
                sc[SC_CHAT0] = ch;
                sc[SC_CHAT1] = ch;
            }
            double tau = factor * (double)n * eps * ch;
            if (nrm <= tau || nonfinite) {
                brk = 2;
                beta[j - 1] = 0.0;
                stt->info[IN_STEPS] = j - 1;
                stt->info[IN_BREAK] = nonfinite ? 3 : 2;
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

__device__ __forceinline__ void cp_async8(double* smem_dst, const double* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

struct HalfArgs {
    rbf_dev_state* stt;
    int64_t n;
    int chunks;
    const double* part;   // product partials [chunks][n]
    const float* part32;  // or FP32 slots [chunks][n] (unscaled FP32 runs), null otherwise
    double slot_scale;    // scale of the FP32 slots (1 or 1/c)
    int side;             // 0: r-side (beta_j), 1: p-side (alpha_j)
    int j;                // 1-based step
    int resume;           // first r-side of a resumed run: scalars are preset
    double factor;        // breakdown factor
    double* alpha;
    double* beta;
    const double* u;      // z_{j-1} (r-side, j >= 2) or w_j (p-side)
    const double* q_raw;  // vector whose norm is finalised here
    double* basis_out;    // w_j (r-side) or z_j (p-side) = q_raw / nrm
    double* v;            // new vector
    float* v32;           // FP32 copy of v (mixed precision) or null
    const double* Q;      // basis to reorthogonalize against (Z or W)
    int64_t ldq;
    int mcount;
    double* hpart;        // [mcount][G] dot partials
    double* gpart;        // 2 x [mcount][barrier groups] group sums (by barrier parity)
    int64_t hpart_len;    // elements of hpart and of gpart (bounds-checked build)
    int64_t gpart_len;
    double* npart;        // in: |q_raw|^2 partials; out: |v|^2 partials
    int rmax;             // slab rows held in shared memory (odd: conflict-free strides)
    unsigned* bar;        // barrier counters (see grid_reduce_sync)
    int bar_group;        // CTAs per barrier group
    unsigned epoch0;      // barriers completed on `bar` before this launch
    long long budget;
};

// One half-step of Algorithm 1 after the product: finalize the norm of q_raw
// (alpha_j or beta_j, breakdown test), form v, and reorthogonalize it twice
// against Q (classical Gram-Schmidt), ending with the |v|^2 partials.
//
// The work runs on v' = v / inv (inv = 1 / nrm, or 1 for a resumed run):
// v' = sum(partials) - (nrm / inv) u with nrm / inv = |q_raw|^2 (beta_j for a
// resumed run), so the square root, the division and the breakdown test (one
// thread of the last warp) run beside the partial sums instead of before them;
// Gram-Schmidt is linear in v', and v = v' inv is formed when v is stored.  The CTA's slabs of the
// product partials, u, q_raw and (STAGE) Q are copied to shared memory with
// cp.async; without STAGE the passes read Q from L2.  Partial sums and dot
// products are split over SPLIT threads per row or per basis vector so that
// all warps share the FP64 work.
template <bool STAGE>
__global__ void __launch_bounds__(SL_THREADS) k_half(HalfArgs a) {
    extern __shared__ double dsm[];
    __shared__ double red[UPD_GROUPS * UPD_ROWS];
    __shared__ double acc_s, fu_s, inv_s;
    __shared__ int brk_s;
    rbf_dev_state* stt = a.stt;
    if (*(volatile int*)&stt->info[IN_DONE]) return;
    const Slab s = slab_of(a.n);
    const int RM = a.rmax;
    int R = (int)(s.r1 - s.r0);
    if (!RBF_IN_RANGE(R, RM + 1)) R = RM;  // the slab must fit its shared-memory rows
    const int M = a.mcount;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* Qs = dsm;                                 // [M][RM]   (STAGE)
    double* ps = Qs + (STAGE ? (size_t)M * RM : 0);   // [chunks][RM] (FP32 slots: half of it)
    double* vs = ps + (a.part32 ? ((size_t)a.chunks * RM + 1) / 2 : (size_t)a.chunks * RM);  // [RM]  v' of the slab
    double* us = vs + RM;                             // [RM]  u of the slab
    double* qs = us + RM;                             // [RM]  q_raw of the slab
    double* r4 = qs + RM;                             // [SPLIT][RM]  (partial sums only)
    double* d4 = r4;                                  // [SPLIT][M]   (passes only: shares r4's space)
    double* hs = d4 + (size_t)SPLIT * M;              // [M]   Q^T v'
    // ---- stage the slab's product partials, u, q_raw and (STAGE) its rows of Q
    if (a.part32) {
        float* ps32 = (float*)ps;
        for (int q = warp; q < a.chunks; q += SL_WARPS)
            for (int i = lane; i < R; i += 32)
                cp_async4(ps32 + (size_t)q * RM + i, a.part32 + (int64_t)q * a.n + s.r0 + i);
    } else {
        for (int q = warp; q < a.chunks; q += SL_WARPS)
            for (int i = lane; i < R; i += 32) cp_async8(ps + (size_t)q * RM + i, a.part + (int64_t)q * a.n + s.r0 + i);
    }
    for (int i = threadIdx.x; i < R; i += SL_THREADS) {
        if (a.u) cp_async8(us + i, a.u + s.r0 + i);
        cp_async8(qs + i, a.q_raw + s.r0 + i);
    }
    if (STAGE)
        for (int m = warp; m < M; m += SL_WARPS)
            for (int i = lane; i < R; i += 32)
                cp_async8(Qs + (size_t)m * RM + i, a.Q + (int64_t)m * a.ldq + s.r0 + i);
    // ---- |q_raw|^2 (every CTA sums the previous partials in the same order)
    if (warp == 0) {
        double acc = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) acc += a.npart[b];
        acc = warp_sum(acc);
        if (lane == 0) {
            acc_s = acc;
            fu_s = a.resume ? stt->scal[SC_BETA] : acc;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // ---- norm, inverse and breakdown test: one thread of the last warp
    if (threadIdx.x == SL_THREADS - 32) {
        double* sc = stt->scal;
        const double eps = DBL_EPSILON;
        double nrm = sqrt(acc_s);
        int brk = 0;
        // c_hat double buffer: the r-side of step j reads slot j&1, writes (j+1)&1;
        // the p-side of step j reads slot (j+1)&1
        const int rd = a.side == 0 ? (a.j & 1) : ((a.j + 1) & 1);
        const double ch_old = sc[SC_CHAT0 + rd];
        double ch_new = ch_old;
        if (a.resume) {
            nrm = sc[SC_BETA];
        } else if (a.side == 1) {
            brk = nrm <= a.factor * (double)a.n * eps * fmax(ch_old, nrm) ? 1 : 0;
        } else if (a.j == 1) {
            brk = nrm > 0.0 ? 0 : 1;
        } else {
            ch_new = fmax(ch_old, hypot(a.alpha[a.j - 2], nrm));
            brk = nrm <= a.factor * (double)a.n * eps * ch_new ? 2 : 0;
        }
        // a norm that is not finite stops the run like a breakdown of the same
        // side (code 3): NaN or Inf in f, the nodes or the operator
        const bool nonfinite = !isfinite(nrm);
        if (nonfinite) brk = (a.side == 1 || a.j == 1) ? 1 : 2;
        inv_s = a.resume ? 1.0 : 1.0 / nrm;
        brk_s = brk;
        if (blockIdx.x == 0) {
            if (a.side == 0 && !a.resume && !nonfinite) sc[SC_CHAT0 + ((a.j + 1) & 1)] = ch_new;
            if (brk) {
                stt->info[IN_STEPS] = a.j - 1;
                stt->info[IN_BREAK] = nonfinite ? 3 : brk;
                if (brk == 2) a.beta[a.j - 1] = 0.0;
                stt->info[IN_DONE] = 1;
            } else if (a.side == 1) {
                a.alpha[a.j - 1] = nrm;
                sc[SC_ALPHA] = nrm;
            } else {
                a.beta[a.j - 1] = nrm;
                sc[SC_BETA] = nrm;
                stt->info[IN_STEPS] = a.j - 1;
            }
        }
    }
    // ---- R1: v' = (sum of partials) - fu u: FP64 partials split SPLIT ways;
    // FP32 slots added in order by a compensated (Neumaier) FP32 sum, hi + lo
    // carried to FP64 and scaled
    const double fu = fu_s;
    if (a.part32) {
        const float* ps32 = (const float*)ps;
        for (int i = threadIdx.x; i < R; i += SL_THREADS) {
            float hi = 0.f, lo = 0.f;
            for (int q = 0; q < a.chunks; ++q) {
                const float t = ps32[(size_t)q * RM + i];
                const float sm = hi + t;
                lo += fabsf(hi) >= fabsf(t) ? (hi - sm) + t : (t - sm) + hi;
                hi = sm;
            }
            double v = ((double)hi + (double)lo) * a.slot_scale;
            if (a.u) v = fma(-fu, us[i], v);
            vs[i] = v;
        }
    } else {
        for (int p = threadIdx.x; p < SPLIT * R; p += SL_THREADS) {
            const int i = p % R, k = p / R;
            double t0 = 0.0, t1 = 0.0;
            int q = k;
            for (; q + SPLIT < a.chunks; q += 2 * SPLIT) {
                t0 += ps[(size_t)q * RM + i];
                t1 += ps[(size_t)(q + SPLIT) * RM + i];
            }
            if (q < a.chunks) t0 += ps[(size_t)q * RM + i];
            r4[(size_t)k * RM + i] = t0 + t1;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < R; i += SL_THREADS) {
            double v = (r4[i] + r4[RM + i]) + (r4[2 * RM + i] + r4[3 * RM + i]);
            if (a.u) v = fma(-fu, us[i], v);
            vs[i] = v;
        }
    }
    __syncthreads();
    if (brk_s) {
        if (brk_s == 2 && a.basis_out)  // w_j = 0 after a beta breakdown
            for (int64_t i = s.r0 + threadIdx.x; i < s.r1; i += SL_THREADS) a.basis_out[i] = 0.0;
        return;
    }
    const double inv = inv_s;
    for (int i = threadIdx.x; i < R; i += SL_THREADS) a.basis_out[s.r0 + i] = qs[i] * inv;
    if (M > 0) {
        const double* qb = STAGE ? (const double*)Qs : a.Q + s.r0;
        const int64_t qld = STAGE ? (int64_t)RM : a.ldq;
        for (int pass = 0; pass < 2; ++pass) {
            // per-slab partials of Q^T v': SPLIT threads per basis vector (rows k, k+SPLIT, ...)
            for (int p = threadIdx.x; p < SPLIT * M; p += SL_THREADS) {
                const int m = p % M, k = p / M;
                const double* q = qb + (int64_t)m * qld;
                double c0 = 0.0, c1 = 0.0;
                int i = k;
                for (; i + SPLIT < R; i += 2 * SPLIT) {
                    c0 = fma(q[i], vs[i], c0);
                    c1 = fma(q[i + SPLIT], vs[i + SPLIT], c1);
                }
                if (i < R) c0 = fma(q[i], vs[i], c0);
                d4[(size_t)k * M + m] = c0 + c1;
            }
            __syncthreads();
            for (int m = threadIdx.x; m < M; m += SL_THREADS) {
                const int64_t hi = (int64_t)m * gridDim.x + blockIdx.x;
                if (RBF_IN_RANGE(hi, a.hpart_len)) a.hpart[hi] = (d4[m] + d4[M + m]) + (d4[2 * M + m] + d4[3 * M + m]);
            }
            // hs = Q^T v': one grid barrier that also sums the partials (fixed order)
            if (!grid_reduce_sync(stt, a.bar, a.bar_group, a.budget, a.epoch0 + pass + 1, a.hpart, a.gpart, hs, M,
                                  a.gpart_len))
                return;
            // v' -= Q hs: thread (row, group of basis vectors), two chains each
            const int row = threadIdx.x % UPD_ROWS;
            const int grp = threadIdx.x / UPD_ROWS;
            for (int base = 0; base < R; base += UPD_ROWS) {
                const int i = base + row;
                double c0 = 0.0, c1 = 0.0;
                if (i < R) {
                    const double* q = qb + i;
                    int m = grp;
                    for (; m + UPD_GROUPS < M; m += 2 * UPD_GROUPS) {
                        c0 = fma(q[(int64_t)m * qld], hs[m], c0);
                        c1 = fma(q[(int64_t)(m + UPD_GROUPS) * qld], hs[m + UPD_GROUPS], c1);
                    }
                    for (; m < M; m += UPD_GROUPS) c0 = fma(q[(int64_t)m * qld], hs[m], c0);
                }
                red[grp * UPD_ROWS + row] = c0 + c1;
                __syncthreads();
                if (grp == 0 && i < R) {
                    double t = 0.0;
#pragma unroll
                    for (int gq = 0; gq < UPD_GROUPS; ++gq) t += red[gq * UPD_ROWS + row];
                    vs[i] -= t;
                }
                __syncthreads();
            }
        }
    } else if (!grid_reduce_sync(stt, a.bar, a.bar_group, a.budget, a.epoch0 + 1, a.hpart, a.gpart, hs, 0,
                                 a.gpart_len)) {
        // nothing to reorthogonalize against: a plain barrier, so that no CTA
        // overwrites npart below while another still reads it above
        return;
    }
    // ---- store v = v' inv (+ FP32 copy) and the |v|^2 partials
    double acc = 0.0;
    for (int i = threadIdx.x; i < R; i += SL_THREADS) {
        const double t = vs[i] * inv;
        a.v[s.r0 + i] = t;
        if (a.v32) a.v32[s.r0 + i] = (float)t;
        acc = fma(t, t, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < SL_WARPS; ++w) t += red[w];
        a.npart[blockIdx.x] = t;
    }
}

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
        stt->scal[SC_CHAT1] = c_hat;
        if (resume) {
            stt->scal[SC_BETA] = beta_now;
            stt->scal[SC_INV_BETA] = 1.0;  // q_raw is the stored, already normalised w
        }
    }
}

}  // namespace

// dynamic shared memory of the half-step kernel when the Q slab is staged:
// the 227 KB a CTA may opt into, less about 2 KB of static shared memory
constexpr size_t HALF_SMEM_STAGE_MAX = 224 * 1024;

// Dynamic shared memory up to which the half-step kernel stages its Q slab.  A
// context whose work runs on several lanes (rbf_gkb_many) keeps each half-step
// CTA small enough that one CTA of every lane fits on an SM at once, so that
// the lanes' cooperative grids can always be resident together.
static size_t half_stage_limit(const rbf_ctx* ctx) {
    const int lanes = ctx->owner ? ctx->owner->lane_count : 1;
    if (lanes <= 1) return HALF_SMEM_STAGE_MAX;
    return (size_t)200 * 1024 / (size_t)lanes - 4 * 1024;
}

static size_t half_smem_bytes(bool stage, int mcount, int chunks, int rmax, bool f32slots) {
    const size_t scratch = std::max((size_t)SPLIT * rmax, (size_t)(SPLIT + 1) * mcount);
    const size_t slots = f32slots ? ((size_t)chunks * rmax + 1) / 2 : (size_t)chunks * rmax;
    return ((stage ? (size_t)mcount * rmax : 0) + slots + (size_t)3 * rmax + scratch) * sizeof(double);
}

static int slab_grid(const rbf_ctx* ctx, int64_t n) {
    int64_t g = ctx->sm_count;
    int64_t need = (n + SL_MAX_ROWS - 1) / SL_MAX_ROWS;
    if (g < need) g = need;
    if (g > n) g = n;
    return (int)(g < 1 ? 1 : g);
}

static int product_chunks(const rbf_ctx* ctx, const rbf_operator* op, int trans) {
    if (op->storage == RBF_MATRIX_FREE) return mf_chunks(ctx, op);
    return trans ? gemv_t_chunks(ctx, op) : gemv_n_chunks(ctx, op);
}

size_t gkb_ws_bytes(const rbf_ctx* ctx, int64_t n, int steps, int precision) {
    (void)precision;
    rbf_operator fake{};
    fake.n = n;
    fake.storage = RBF_MATRIX_FREE;
    fake.precision = RBF_MIXED;
    int ch = mf_part_rows(ctx, &fake);
    fake.precision = RBF_FP64;
    ch = std::max(ch, mf_part_rows(ctx, &fake));
    fake.storage = RBF_ASSEMBLED;
    for (int prec : {RBF_MIXED, RBF_FP64}) {  // the assembled products' partial-sum rows
        fake.precision = prec;
        ch = std::max(ch, std::max(gemv_t_chunks(ctx, &fake), gemv_n_chunks(ctx, &fake)));
    }
    ch = std::max(ch, 8);  // the fixed-point A z (flat split: at most 8 pieces per row)
    const int G = slab_grid(ctx, n);
    size_t b = 0;
    b += ws_align((size_t)ch * n * 8);                // partials
    b += 2 * ws_align((size_t)n * 8);                 // vr, vp
    b += 2 * ws_align((size_t)n * 4);                 // vr32, vp32
    b += ws_align((size_t)3 * n * 4);                 // FP32 node coordinates (matrix-free FP32)
    b += ws_align((size_t)(steps + 2) * G * 8);       // hpart
    b += ws_align((size_t)2 * (steps + 2) * G * 8);   // gpart (two buffers, at most G groups)
    b += ws_align((size_t)(G + 2) * BAR_STRIDE * 4);  // barrier counters
    b += ws_align((size_t)G * 8);                     // npart
    return b + 4096;
}

// Launch the product "part = M q_raw" for one half-step.
// fx: the run's fixed-point copies of A (FP64 assembled operators), or null.
static rbf_status gkb_product(rbf_ctx* ctx, const rbf_operator* op, int trans, const double* q_raw,
                              const float* q32, const float* X32, const FxCopies* fx, double* part,
                              const int* done) {
    const int slot = rbf_prod_begin(ctx, trans);
    rbf_status st;
    if (op->storage == RBF_MATRIX_FREE) st = launch_mf_partial(ctx, op, trans, q_raw, q32, X32, part, done);
    else if (fx) st = trans ? launch_fx_t(ctx, op, *fx, q_raw, part, done) : launch_fx_n(ctx, op, *fx, q_raw, part, done);
    else if (trans) st = launch_gemv_t_partial(ctx, op, q_raw, q32, part, done);
    else st = launch_gemv_n(ctx, op, q_raw, q32, part, done);
    rbf_prod_end(ctx, trans, slot);
    return st;
}

// Workspace of one GKB run on op: the fixed-point copies of A are included
// (*fx = true) when the operator takes them and they fit under the cap.
static size_t run_ws_bytes(const rbf_ctx* ctx, const rbf_operator* op, int capacity, bool* fx) {
    const size_t base = gkb_ws_bytes(ctx, op->n, capacity, op->precision);
    *fx = fx_eligible(ctx, op);
    if (*fx) {
        const size_t full = base + fx_ws_bytes(op);
        if (ctx->opt.workspace_cap > 0 && full > (size_t)ctx->opt.workspace_cap) *fx = false;
        else return full;
    }
    return base;
}

// One GKB run split into its launch sequence, so that several independent runs
// can be enqueued step by step on different streams (rbf_gkb_many): begin()
// prepares the workspace and the first r-side input, step(j) enqueues the
// four launches of step j, end() closes with beta_{l+1} and w_{l+1}.  Nothing
// here synchronises except the resume path, which reads beta_{j_begin}.
struct GkbRun {
    rbf_ctx* ctx = nullptr;
    const rbf_operator* op = nullptr;
    rbf_gkb_state* st = nullptr;
    int64_t n = 0;
    int G = 0, chT = 0, chN = 0, rmax = 0, bar_group = 0, bar_k = 0, j_begin = 1;
    double *part = nullptr, *vr = nullptr, *vp = nullptr, *hpart = nullptr, *gpart = nullptr, *npart = nullptr;
    float *vr32 = nullptr, *vp32 = nullptr, *X32 = nullptr;  // X32: FP32 node coordinates (matrix-free FP32)
    FxCopies fx;              // fixed-point copies of A (use_fx)
    bool use_fx = false;
    bool f32slots = false;    // the products' partials are FP32 slots (mf_slots_f32)
    double slot_scale = 1.0;  // their scale
    unsigned* bar = nullptr;
    const double* q_raw = nullptr;
    unsigned epochs = 0;  // barriers on `bar` since it was zeroed
    bool mixed = false;

    rbf_status begin(rbf_ctx* c, const rbf_operator* o, const double* f, int jb, rbf_gkb_state* s_) {
        ctx = c;
        op = o;
        st = s_;
        j_begin = jb;
        n = op->n;
        G = slab_grid(ctx, n);
        if ((n + G - 1) / G > SL_MAX_ROWS) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "n too large for slab kernels");
        if (st->capacity + 1 > 1024) return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "capacity above 1023 steps");
        {
            const size_t need = run_ws_bytes(ctx, op, st->capacity, &use_fx);
            const rbf_status e = rbf_ws_reserve(ctx, need);
            if (e != RBF_OK) {
                if (!use_fx) return e;
                use_fx = false;  // no room for the fixed-point copies: FP64 FMA products
                RBF_TRY(rbf_ws_reserve(ctx, gkb_ws_bytes(ctx, n, st->capacity, op->precision)));
            }
        }
        WsCarve wc(ctx->ws);
        chT = product_chunks(ctx, op, 1);
        chN = use_fx ? fx_n_chunks(ctx, n) : product_chunks(ctx, op, 0);
        f32slots = mf_slots_f32(ctx, op);
        slot_scale = op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0;
        const int prow = op->storage == RBF_MATRIX_FREE ? mf_part_rows(ctx, op) : 0;
        part = wc.take<double>((size_t)std::max(prow, std::max(chT, chN)) * n);
        vr = wc.take<double>((size_t)n);
        vp = wc.take<double>((size_t)n);
        vr32 = wc.take<float>((size_t)n);
        vp32 = wc.take<float>((size_t)n);
        if (op->storage == RBF_MATRIX_FREE && op->precision != RBF_FP64) {
            X32 = wc.take<float>((size_t)3 * n);
            RBF_TRY(launch_to_f32(ctx, 3 * n, op->d_nodes, X32));
        }
        hpart = wc.take<double>((size_t)(st->capacity + 2) * G);
        bar_group = 1;
        while (bar_group * bar_group < G) ++bar_group;
        bar_k = (G + bar_group - 1) / bar_group;
        gpart = wc.take<double>((size_t)2 * (st->capacity + 2) * G);
        bar = wc.take<unsigned>((size_t)(bar_k + 2) * BAR_STRIDE);
        cudaStream_t s = ctx->stream;
        RBF_CUDA(ctx, cudaMemsetAsync(bar, 0, (size_t)(bar_k + 2) * BAR_STRIDE * sizeof(unsigned), s));
        // shared-memory plan of the half-step kernel: stage the Q slab when it fits
        rmax = (int)((n + G - 1) / G) | 1;
        const int chmax = chT > chN ? chT : chN;
        // The Q slab is staged in every half-step whose slab fits (mcount grows with
        // the step, so long runs on large N stage their early steps only); the
        // unstaged kernel must fit for the largest basis.
        {
            const size_t need = half_smem_bytes(false, st->capacity + 1, chmax, rmax, f32slots);
            if (need > HALF_SMEM_STAGE_MAX)
                return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "half-step shared memory too large (%zu bytes)", need);
            if (need > 48 * 1024)
                RBF_CUDA(ctx, cudaFuncSetAttribute((const void*)k_half<false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
            RBF_CUDA(ctx, cudaFuncSetAttribute((const void*)k_half<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)HALF_SMEM_STAGE_MAX));
        }
        npart = wc.take<double>((size_t)G);
        if (use_fx) {
            fx = fx_carve(wc, op);
            RBF_TRY(launch_fx_prepare(ctx, op, fx));
        }
        mixed = op->precision == RBF_MIXED;
        rbf_dev_state* dst = ctx->d_state;
        epochs = 0;
        // q_raw for the first r-side: f (fresh run) or the stored w_{j_begin} (resume)
        q_raw = vp;
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
            const double* w = st->d_W + (int64_t)(j_begin - 1) * st->ldw;
            k_norm_partials<<<G, SL_THREADS, 0, s>>>(n, w, npart, vp, mixed ? vp32 : nullptr);
            RBF_LAUNCHED(ctx, "k_norm_partials");
        }
        return RBF_OK;
    }

    rbf_status half(int side, int j, int resume, const double* u, const double* qr, double* bout, double* v,
                    float* v32, const double* Q, int64_t ldq, int mcount, int chunks) {
        HalfArgs a;
        a.stt = ctx->d_state;
        a.n = n;
        a.chunks = chunks;
        a.part = part;
        a.part32 = f32slots ? (const float*)part : nullptr;
        a.slot_scale = slot_scale;
        a.side = side;
        a.j = j;
        a.resume = resume;
        a.factor = ctx->opt.breakdown_factor;
        a.alpha = st->d_alpha;
        a.beta = st->d_beta;
        a.u = u;
        a.q_raw = qr;
        a.basis_out = bout;
        a.v = v;
        a.v32 = v32;
        a.Q = Q;
        a.ldq = ldq;
        a.mcount = mcount;
        a.hpart = hpart;
        a.gpart = gpart;
        a.hpart_len = (int64_t)(st->capacity + 2) * G;
        a.gpart_len = (int64_t)2 * (st->capacity + 2) * G;
        a.npart = npart;
        a.rmax = rmax;
        a.bar = bar;
        a.bar_group = bar_group;
        a.epoch0 = epochs;
        a.budget = ctx->opt.wait_budget;
        void* args[] = {&a};
        const bool stage = half_smem_bytes(true, mcount, chunks, rmax, f32slots) <= half_stage_limit(ctx);
        const size_t smem = half_smem_bytes(stage, mcount, chunks, rmax, f32slots);
        const int slot = rbf_prod_begin(ctx, 2);
        cudaError_t e = cudaLaunchCooperativeKernel(stage ? (const void*)k_half<true> : (const void*)k_half<false>,
                                                    dim3(G), dim3(SL_THREADS), args, smem, ctx->stream);
        rbf_prod_end(ctx, 2, slot);
        ctx->launches++;
        if (e != cudaSuccess)
            return rbf_fail(ctx, RBF_ERR_CUDA, "cooperative launch of k_half failed: %s", cudaGetErrorString(e));
        epochs += mcount > 0 ? 2 : 1;  // two reorthogonalization barriers, or one plain barrier
        return RBF_OK;
    }

    rbf_status step(int j) {
        const int* done = &ctx->d_state->info[IN_DONE];
        double* W = st->d_W;
        double* Z = st->d_Z;
        const int64_t ldw = st->ldw, ldz = st->ldz;
        // ---------------- r-side: r = A^T w_j - beta_j z_{j-1} ----------------
        RBF_TRY(gkb_product(ctx, op, 1, q_raw, vp32, X32, use_fx ? &fx : nullptr, part, done));
        RBF_TRY(half(0, j, (j == j_begin && j_begin > 1) ? 1 : 0, j >= 2 ? Z + (int64_t)(j - 2) * ldz : nullptr,
                     q_raw, W + (int64_t)(j - 1) * ldw, vr, mixed ? vr32 : nullptr, Z, ldz, j - 1, chT));
        // ---------------- p-side: p = A z_j - alpha_j w_j ----------------
        RBF_TRY(gkb_product(ctx, op, 0, vr, vr32, X32, use_fx ? &fx : nullptr, part, done));
        RBF_TRY(half(1, j, 0, W + (int64_t)(j - 1) * ldw, vr, Z + (int64_t)(j - 1) * ldz, vp,
                     mixed ? vp32 : nullptr, W, ldw, j, chN));
        q_raw = vp;
        return RBF_OK;
    }

    rbf_status end(int j_end) {
        cudaStream_t s = ctx->stream;
        double* wl = st->d_W + (int64_t)j_end * st->ldw;
        // beta_{l+1} and w_{l+1}
        k_finalize<<<1, 256, 0, s>>>(ctx->d_state, npart, G, 0, j_end + 1, n, ctx->opt.breakdown_factor,
                                     st->d_alpha, st->d_beta, wl, 1);
        RBF_LAUNCHED(ctx, "k_finalize");
        k_write_basis<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctx->d_state, n, SC_INV_BETA, vp, wl);
        RBF_LAUNCHED(ctx, "k_write_basis");
        return RBF_OK;
    }
};

rbf_status gkb_run(rbf_ctx* ctx, const rbf_operator* op, const double* f, int j_begin, int j_end,
                   rbf_gkb_state* st) {
    GkbRun r;
    RBF_TRY(r.begin(ctx, op, f, j_begin, st));
    for (int j = j_begin; j <= j_end; ++j) RBF_TRY(r.step(j));
    return r.end(j_end);
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
    st->c_hat = ctx->h_state->scal[SC_CHAT0] > ctx->h_state->scal[SC_CHAT1] ? ctx->h_state->scal[SC_CHAT0]
                                                                           : ctx->h_state->scal[SC_CHAT1];
    RBF_TRY(rbf_check_all(ctx));
    if (ctx->h_state->info[IN_ERR] != 0)
        return rbf_fail(ctx, (rbf_status)ctx->h_state->info[IN_ERR],
                        "a bounded device-side wait gave up (grid barrier of the GKB half-step)");
    return RBF_OK;
}

extern "C" rbf_status rbf_gkb(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int steps,
                              rbf_gkb_state* st) {
    RbfRange range_("rbf_gkb");
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
    RbfRange range_("rbf_gkb_resume");
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

// Several independent GKB runs, spread over lanes (child contexts with their
// own streams) and enqueued one step at a time per lane, so that one run's
// latency-bound half-step kernels and launch gaps overlap another run's
// products.  Each lane runs its share of the runs one after another.
extern "C" rbf_status rbf_gkb_many(rbf_ctx* ctx, int count, const rbf_operator* ops, const double* const* d_f,
                                   int steps, rbf_gkb_state* states, int lanes, int assemble) {
    RbfRange range_("rbf_gkb_many");
    if (!ctx) return RBF_ERR_INVALID;
    if (count < 1 || !ops || !d_f || !states) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_gkb_many: bad arguments");
    if (lanes < 0 || lanes > rbf_ctx::MAX_LANES)
        return rbf_fail(ctx, RBF_ERR_INVALID, "lanes must be 0 (default) or 1..%d", rbf_ctx::MAX_LANES);
    for (int i = 0; i < count; ++i) {
        if (!d_f[i]) return rbf_fail(ctx, RBF_ERR_INVALID, "d_f[%d] is NULL", i);
        RBF_TRY(check_state(ctx, &ops[i], &states[i], steps));
    }
    int L = lanes == 0 ? rbf_ctx::MAX_LANES : lanes;
    if (L > count) L = count;
    // every lane's half-step grid must fit on the SMs beside the other lanes'
    // (they are cooperative and wait for one another's CTAs only within a grid)
    for (int i = 0; i < count && L > 1; ++i) {
        const int64_t n = ops[i].n;
        const int G = slab_grid(ctx, n);
        const int rmax = (int)((n + G - 1) / G) | 1;
        int chmax = std::max(product_chunks(ctx, &ops[i], 0), product_chunks(ctx, &ops[i], 1));
        if (fx_eligible(ctx, &ops[i])) chmax = std::max(chmax, fx_n_chunks(ctx, n));
        const size_t need = half_smem_bytes(false, states[i].capacity + 1, chmax, rmax, mf_slots_f32(ctx, &ops[i]));
        if (need > HALF_SMEM_STAGE_MAX) continue;  // the run itself is refused with RBF_ERR_UNSUPPORTED below
        int per_sm = 0;
        if (need > 48 * 1024)
            RBF_CUDA(ctx, cudaFuncSetAttribute((const void*)k_half<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)need));
        RBF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_half<false>, SL_THREADS,
                                                                    need));
        const int64_t fit = (int64_t)per_sm * ctx->sm_count / G;
        if (fit < L) L = fit < 1 ? 1 : (int)fit;
    }
    ctx->lane_count = L;
    RBF_TRY(rbf_many_slots(ctx, count));
    // operators that differ only in k are assembled two at a time on the
    // context stream (the distances and 1/sqrt(s) computed once), before the
    // lanes start; the others by their lane
    std::vector<char> assembled(count, 0);
    if (assemble)
        for (int i = 0; i < count; ++i)
            for (int j = i + 1; j < count && !assembled[i]; ++j)
                if (!assembled[j] && assemble_pairable(&ops[i], &ops[j])) {
                    RBF_TRY(launch_assemble_pair(ctx, &ops[i], &ops[j]));
                    assembled[i] = assembled[j] = 1;
                }
    RBF_TRY(rbf_lanes_fork(ctx, L));
    rbf_timer_start(ctx);
    std::vector<rbf_ctx*> lane(L);
    for (int l = 0; l < L; ++l) RBF_TRY(rbf_lane(ctx, l, &lane[l]));
    // workspace sized once per lane for the largest of its runs (growing it
    // between runs would synchronise the lane)
    // (with the fixed-point copies of A where they fit; a lane without room
    // for them runs its FP64 assembled products with FMAs, see GkbRun::begin)
    for (int l = 0; l < L; ++l) {
        size_t need = 0, base = 0;
        for (int i = l; i < count; i += L) {
            bool fx_i = false;
            need = std::max(need, run_ws_bytes(lane[l], &ops[i], states[i].capacity, &fx_i));
            base = std::max(base, gkb_ws_bytes(lane[l], ops[i].n, states[i].capacity, ops[i].precision));
        }
        rbf_status e = rbf_ws_reserve(lane[l], need);
        if (e != RBF_OK && need > base) e = rbf_ws_reserve(lane[l], base);
        if (e != RBF_OK) {
            rbf_lanes_join(ctx, L);
            return rbf_fail(ctx, e, "lane %d: %s", l, rbf_last_error(lane[l]));
        }
    }
    std::vector<GkbRun> run(count);
    std::vector<int> cur(L), jnext(L, 0);  // lane l: its current run and the next step (0 = not begun)
    for (int l = 0; l < L; ++l) cur[l] = l;
    rbf_status err = RBF_OK;
    for (bool busy = true; busy && err == RBF_OK;) {
        busy = false;
        for (int l = 0; l < L && err == RBF_OK; ++l) {
            const int i = cur[l];
            if (i >= count) continue;
            busy = true;
            rbf_ctx* c = lane[l];
            if (jnext[l] == 0) {
                if (assemble && ops[i].storage == RBF_ASSEMBLED && !assembled[i]) err = launch_assemble(c, &ops[i]);
                if (err == RBF_OK) err = run[i].begin(c, &ops[i], d_f[i], 1, &states[i]);
                jnext[l] = 1;
            }
            if (err == RBF_OK) err = run[i].step(jnext[l]++);
            if (err == RBF_OK && jnext[l] > steps) {
                err = run[i].end(steps);
                if (err == RBF_OK) {
                    cudaError_t e = cudaMemcpyAsync(&ctx->h_many[i], c->d_state, sizeof(rbf_dev_state),
                                                    cudaMemcpyDeviceToHost, c->stream);
                    if (e != cudaSuccess)
                        err = rbf_fail(c, RBF_ERR_CUDA, "state copy failed: %s", cudaGetErrorString(e));
                }
                cur[l] += L;
                jnext[l] = 0;
            }
            if (err != RBF_OK) rbf_fail(ctx, err, "lane %d, run %d: %s", l, i, rbf_last_error(c));
        }
    }
    rbf_status je = rbf_lanes_join(ctx, L);
    if (err != RBF_OK) return err;
    RBF_TRY(je);
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RBF_CUDA(ctx, cudaGetLastError());
    RBF_TRY(rbf_check_all(ctx));
    int total = 0;
    for (int i = 0; i < count; ++i) {
        const rbf_dev_state& h = ctx->h_many[i];
        states[i].steps_done = h.info[IN_STEPS];
        states[i].breakdown = h.info[IN_BREAK];
        states[i].c_hat = std::max(h.scal[SC_CHAT0], h.scal[SC_CHAT1]);
        total += states[i].steps_done;
        if (h.info[IN_ERR] != 0)
            return rbf_fail(ctx, (rbf_status)h.info[IN_ERR],
                            "run %d: a bounded device-side wait gave up (grid barrier of the GKB half-step)", i);
    }
    ctx->tim.gkb_ms = rbf_timer_stop(ctx);
    ctx->tim.gkb_steps = total;
    return RBF_OK;
}

// Host snapshot of a GKB state (checkpoint/resume through host memory): the
// first l+1 columns of W, l of Z, alpha[l] and beta[l+1], packed with leading
// dimension n on the host.
extern "C" rbf_status rbf_gkb_snapshot(rbf_ctx* ctx, const rbf_gkb_state* st, double* h_W, double* h_Z,
                                       double* h_alpha, double* h_beta) {
    RbfRange range_("rbf_gkb_snapshot");
    if (!ctx) return RBF_ERR_INVALID;
    if (!st || !h_W || !h_Z || !h_alpha || !h_beta || !st->d_W || !st->d_Z || !st->d_alpha || !st->d_beta)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_gkb_snapshot: NULL argument");
    const int l = st->steps_done;
    const int64_t n = st->n;
    if (l < 0 || l > st->capacity || n < 1 || st->ldw < n || st->ldz < n)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_gkb_snapshot: inconsistent state");
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaMemcpy2DAsync(h_W, n * sizeof(double), st->d_W, st->ldw * sizeof(double), n * sizeof(double),
                                    (size_t)l + 1, cudaMemcpyDeviceToHost, s));
    if (l > 0) {
        RBF_CUDA(ctx, cudaMemcpy2DAsync(h_Z, n * sizeof(double), st->d_Z, st->ldz * sizeof(double),
                                        n * sizeof(double), (size_t)l, cudaMemcpyDeviceToHost, s));
        RBF_CUDA(ctx, cudaMemcpyAsync(h_alpha, st->d_alpha, (size_t)l * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    RBF_CUDA(ctx, cudaMemcpyAsync(h_beta, st->d_beta, ((size_t)l + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    return RBF_OK;
}

extern "C" rbf_status rbf_gkb_restore(rbf_ctx* ctx, rbf_gkb_state* st, const double* h_W, const double* h_Z,
                                      const double* h_alpha, const double* h_beta, int steps_done, int breakdown,
                                      double c_hat) {
    RbfRange range_("rbf_gkb_restore");
    if (!ctx) return RBF_ERR_INVALID;
    if (!st || !h_W || !h_Z || !h_alpha || !h_beta || !st->d_W || !st->d_Z || !st->d_alpha || !st->d_beta)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_gkb_restore: NULL argument");
    const int l = steps_done;
    const int64_t n = st->n;
    if (l < 1 || l > st->capacity || n < 1 || st->ldw < n || st->ldz < n || breakdown < 0 || breakdown > 3 ||
        !(c_hat >= 0.0))
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_gkb_restore: steps_done outside [1, capacity] or bad scalars");
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaMemcpy2DAsync(st->d_W, st->ldw * sizeof(double), h_W, n * sizeof(double), n * sizeof(double),
                                    (size_t)l + 1, cudaMemcpyHostToDevice, s));
    RBF_CUDA(ctx, cudaMemcpy2DAsync(st->d_Z, st->ldz * sizeof(double), h_Z, n * sizeof(double), n * sizeof(double),
                                    (size_t)l, cudaMemcpyHostToDevice, s));
    RBF_CUDA(ctx, cudaMemcpyAsync(st->d_alpha, h_alpha, (size_t)l * sizeof(double), cudaMemcpyHostToDevice, s));
    RBF_CUDA(ctx, cudaMemcpyAsync(st->d_beta, h_beta, ((size_t)l + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
    RBF_CUDA(ctx, cudaStreamSynchronize(s));  // the host arrays may be released on return
    st->steps_done = l;
    st->breakdown = breakdown;
    st->c_hat = c_hat;
    return RBF_OK;
}

RBF_CHECK_READER(gkb)
