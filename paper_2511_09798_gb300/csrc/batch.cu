// Batched GKB: many independent collocation problems of uneven size advance
// through Algorithm 1 together (mixed precision: matrix-free FP32 products,
// FP64 reorthogonalization, norms and scalars), then through the projected
// solve of Algorithm 4.
//
// Layout: every per-row vector of the batch is the concatenation of the
// instances' vectors (instance b at off_b = sum_{a<b} n_a, T = sum n_b rows).
// Per step:
//   k_mf_batch<1>   partial sums of A_b^T q_b for all instances: one CTA per
//                   work item (instance, tile pair of node blocks), each node
//                   pair evaluated once for A_ij and A_ji (mf_core.cuh); one
//                   partial slot per block of the instance
//   k_half_batch    cooperative kernel over the T concatenated rows (balanced
//                   slabs, a slab may span several instances): per-instance
//                   norm finalisation and breakdown test, then classical
//                   Gram-Schmidt applied twice against each instance's basis,
//                   with per-instance dot partials reduced across the CTAs that
//                   share the instance (bounded grid barriers)
//   k_mf_batch<0>, k_half_batch   the same for the p-side
// The whole step loop is captured into one CUDA graph and launched once.  The
// block size of the batched product (4 or 8 rows per lane: blocks of 128 or
// 256 nodes) is chosen by timing both on the batch itself the first time a
// batch shape is seen.
#include <algorithm>
#include <cfloat>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "mf_core.cuh"

namespace {

struct BInst {
    int64_t off;        // row offset of the instance in concatenated vectors
    int64_t n, ni;
    float c2, k2;
    double scale;       // 1 (c-form) or 1/c (eps-form)
    int chunks;         // product: partial slots = blocks of the tile-pair product
    int64_t poff;       // product partials offset (chunks * n doubles)
    int cfirst, ncta;   // half-step CTAs whose slabs intersect the instance
    int64_t hoff;       // dot partials offset ((L+2) * ncta doubles)
    int noff;           // norm partials offset (ncta doubles)
};

struct MfItem {  // tile (bi, bj), bi <= bj, of instance b
    int b, bi, bj;
};

constexpr int HB_THREADS = 256;
constexpr int DG_LOG = 2;
constexpr int DG = 1 << DG_LOG;  // basis vectors per warp in the half-step's dot products
constexpr int HB_WARPS = HB_THREADS / 32;
constexpr int SEGMAX = 16;       // instances intersecting one slab
constexpr int UPD_ROWS_B = 64;
constexpr int UPD_GROUPS_B = HB_THREADS / UPD_ROWS_B;


// ---------------------------------------------------------------------------
// Batched matrix-free product: the single-instance tile-pair product
// (mf_core.cuh) over a work list of (instance, tile) items.
// ---------------------------------------------------------------------------
template <int TRANS, int R>
__global__ void __launch_bounds__(MS_W * 32) k_mf_batch(const MfItem* __restrict__ items, const BInst* __restrict__ inst,
                                                      const float* __restrict__ X32_all,
                                                      const float* __restrict__ x32_all, float* __restrict__ part_all,
                                                      const int* __restrict__ done) {
    const MfItem it = items[blockIdx.x];
    if (done && done[it.b]) return;
    const BInst I = inst[it.b];
    // the tile lies inside its instance's block triangle
    if (!RBF_IN_RANGE(it.bj, I.chunks) || !RBF_IN_RANGE(it.bi, it.bj + 1)) return;
    ms_tile_product<TRANS, R, float>(X32_all + 3 * I.off, I.n, I.ni, I.c2, I.k2, I.scale, x32_all + I.off, it.bi,
                                     it.bj, part_all + I.poff);
}

// ---------------------------------------------------------------------------
// Two-level bounded grid barrier (same scheme as the single-instance kernel).
// ---------------------------------------------------------------------------
constexpr int BAR_STRIDE_B = 32;

__device__ bool grid_sync_b(rbf_dev_state* __restrict__ stt, unsigned* __restrict__ bar, int group,
                            long long budget) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int G = gridDim.x;
        const int K = (G + group - 1) / group;
        const int grp = blockIdx.x / group;
        const int members = min(group, G - grp * group);
        unsigned* sub = bar + (size_t)grp * BAR_STRIDE_B;
        unsigned* top = bar + (size_t)K * BAR_STRIDE_B;
        volatile unsigned* gen = bar + (size_t)(K + 1) * BAR_STRIDE_B;
        const unsigned g0 = *gen;
        __threadfence();
        int good = 1;
        if (atomicAdd(sub, 1u) == (unsigned)members - 1) {
            atomicExch(sub, 0u);
            if (atomicAdd(top, 1u) == (unsigned)K - 1) {
                atomicExch(top, 0u);
                __threadfence();
                atomicAdd((unsigned*)gen, 1u);
            }
        }
        long long it = 0;
        while (*gen == g0) {
            if (++it > budget) {
                good = 0;
                atomicExch(&stt->info[IN_ERR], (int)RBF_ERR_TIMEOUT);
                break;
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// per-instance flags, struct of arrays [6][B]
enum { BI_STEPS = 0, BI_BREAK = 1, BI_DONE0 = 2, BI_DONE1 = 3, BI_LIMIT = 4 };

struct HalfBArgs {
    const BInst* inst;
    const int64_t* offs;     // [B+1] cumulative row offsets
    int B;
    int64_t T;
    int L;
    int j;                   // 1-based step
    int side;                // 0: r-side (beta_j), 1: p-side (alpha_j)
    double factor;
    double* alpha_all;       // [B][L]
    double* beta_all;        // [B][L+1]
    double* W_all;           // W_b at (L+1) off_b, ld n_b
    double* Z_all;           // Z_b at L off_b, ld n_b
    const double* qraw_all;  // vector whose norm is finalised
    double* v_all;           // new vector
    float* v32_all;          // its FP32 copy
    const float* part_all;   // product partial slots (FP32 runs, unscaled)
    double* hpart_all;
    double* h_all;           // [B][L+2]
    double* npart_all;       // per-instance norm partials
    int* binfo;              // [6][B]
    const int* done_in;      // done flags before this launch
    int* done_out;           // done flags after this launch
    const int* limit;        // [B] steps per instance (the instance stops after step limit[b])
    double* chat_all;        // [B][2]
    rbf_dev_state* stt;
    unsigned* bar;
    int bar_group;
    long long budget;
    int rmax;
};

__global__ void __launch_bounds__(HB_THREADS, 4) k_half_batch(HalfBArgs a) {
    extern __shared__ double dsm[];
    __shared__ int seg_b[SEGMAX], seg_base[SEGMAX], seg_act[SEGMAX], seg_brk[SEGMAX], seg_stop[SEGMAX];
    __shared__ int64_t seg_i0[SEGMAX], seg_i1[SEGMAX];
    __shared__ double seg_nrm[SEGMAX], seg_inv[SEGMAX];
    __shared__ int nseg, nrows;
    __shared__ double red[UPD_GROUPS_B * UPD_ROWS_B];
    const int G = gridDim.x;
    const int L = a.L;
    const int M = a.side == 0 ? a.j - 1 : a.j;  // basis vectors to orthogonalize against
    double* vs = dsm;                 // [rmax]
    double* hs = dsm + a.rmax;        // [SEGMAX][L+2]
    const int64_t R0 = a.T * blockIdx.x / G, R1 = a.T * (blockIdx.x + 1) / G;
    if (threadIdx.x == 0) {
        int lo = 0, hi = a.B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (a.offs[mid] <= R0) lo = mid; else hi = mid - 1;
        }
        int ns = 0, base = 0;
        for (int b = lo; b < a.B && a.offs[b] < R1 && ns < SEGMAX; ++b) {
            const int64_t i0 = max(R0, a.offs[b]) - a.offs[b];
            const int64_t i1 = min(R1, a.offs[b + 1]) - a.offs[b];
            if (i1 <= i0) continue;
            seg_b[ns] = b;
            seg_i0[ns] = i0;
            seg_i1[ns] = i1;
            seg_base[ns] = base;
            base += (int)(i1 - i0);
            ++ns;
        }
        nseg = ns;
        // the slab's rows must fit the shared-memory vector of rmax rows
        nrows = RBF_IN_RANGE(base, a.rmax + 1) ? base : a.rmax;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- per-instance norm finalisation (warp per segment)
    for (int sx = warp; sx < nseg; sx += HB_WARPS) {
        const int b = seg_b[sx];
        const BInst I = a.inst[b];
        const int active = a.done_in[b] == 0;
        double acc = 0.0;
        for (int q = lane; q < I.ncta; q += 32) acc += a.npart_all[I.noff + q];
        acc = warp_sum(acc);
        if (lane == 0) {
            const double eps = DBL_EPSILON;
            const double nrm = sqrt(acc);
            double* ch = a.chat_all + 2 * b;
            const int rd = a.side == 0 ? (a.j & 1) : ((a.j + 1) & 1);
            const double ch_old = ch[rd];
            double ch_new = ch_old;
            int brk = 0;
            if (active) {
                if (a.side == 1) {
                    brk = nrm <= a.factor * (double)I.n * eps * fmax(ch_old, nrm) ? 1 : 0;
                } else if (a.j == 1) {
                    brk = nrm > 0.0 ? 0 : 1;
                } else {
                    ch_new = fmax(ch_old, hypot(a.alpha_all[(size_t)b * L + a.j - 2], nrm));
                    brk = nrm <= a.factor * (double)I.n * eps * ch_new ? 2 : 0;
                }
            }
            // a norm that is not finite stops the instance like a breakdown of
            // the same side (code 3)
            const bool nonfinite = active && !isfinite(nrm);
            if (nonfinite) {
                brk = (a.side == 1 || a.j == 1) ? 1 : 2;
                ch_new = ch_old;
            }
            // the instance's step limit: step limit[b] + 1 only finalises beta and w
            const int stop = active && !brk && a.side == 0 && a.limit && a.j == a.limit[b] + 1;
            seg_act[sx] = active && !brk && !stop;
            seg_brk[sx] = active ? brk : 0;
            seg_stop[sx] = stop;
            seg_nrm[sx] = nrm;
            seg_inv[sx] = 1.0 / nrm;
            if ((int)blockIdx.x == I.cfirst) {  // the instance's first CTA writes its scalars
                if (active && a.side == 0) ch[(a.j + 1) & 1] = ch_new;
                a.done_out[b] = (!active || brk || stop) ? 1 : 0;
                if (active) {
                    if (brk) {
                        a.binfo[BI_STEPS * a.B + b] = a.j - 1;
                        a.binfo[BI_BREAK * a.B + b] = nonfinite ? 3 : brk;
                        if (brk == 2) a.beta_all[(size_t)b * (L + 1) + a.j - 1] = 0.0;
                    } else if (a.side == 1) {
                        a.alpha_all[(size_t)b * L + a.j - 1] = nrm;
                    } else {
                        a.beta_all[(size_t)b * (L + 1) + a.j - 1] = nrm;
                        a.binfo[BI_STEPS * a.B + b] = a.j - 1;
                    }
                }
            }
        }
    }
    __syncthreads();
    // ---- R1 per segment: v = (sum of partials) / nrm - nrm u; store q_raw / nrm
    for (int sx = 0; sx < nseg; ++sx) {
        const int b = seg_b[sx];
        if (!seg_act[sx] && seg_brk[sx] != 2 && !seg_stop[sx]) continue;
        const BInst I = a.inst[b];
        const int64_t n = I.n;
        double* Wb = a.W_all + (size_t)(L + 1) * I.off;
        double* Zb = a.Z_all + (size_t)L * I.off;
        const double* u = a.side == 0 ? (a.j >= 2 ? Zb + (int64_t)(a.j - 2) * n : nullptr) : Wb + (int64_t)(a.j - 1) * n;
        double* bout = a.side == 0 ? Wb + (int64_t)(a.j - 1) * n : Zb + (int64_t)(a.j - 1) * n;
        const double* qr = a.qraw_all + I.off;
        const float* part = a.part_all + I.poff;
        const double nrm = seg_nrm[sx], inv = seg_inv[sx];
        for (int64_t i = seg_i0[sx] + threadIdx.x; i < seg_i1[sx]; i += HB_THREADS) {
            if (seg_brk[sx] == 2) {  // w_j = 0 after a beta breakdown
                bout[i] = 0.0;
                continue;
            }
            if (seg_stop[sx]) {  // last step of a limited instance: w_j only
                bout[i] = qr[i] * inv;
                continue;
            }
            // the instance's partial slots (one FP32 run per block of the
            // tile-pair product), added in order by a compensated FP32 sum
            // (Neumaier: hi + lo carries the sum to ~2^-48 relative; FP64 adds
            // would cost as much as the reorthogonalization's FMAs here)
            float hi = 0.f, lo = 0.f;
            auto add = [&hi, &lo](float t) {
                const float sm = hi + t;
                lo += fabsf(hi) >= fabsf(t) ? (hi - sm) + t : (t - sm) + hi;
                hi = sm;
            };
            int q = 0;
            for (; q + 3 < I.chunks; q += 4) {  // four loads in flight, added in order
                const float t0 = part[(int64_t)q * n + i], t1 = part[(int64_t)(q + 1) * n + i];
                const float t2 = part[(int64_t)(q + 2) * n + i], t3 = part[(int64_t)(q + 3) * n + i];
                add(t0);
                add(t1);
                add(t2);
                add(t3);
            }
            for (; q < I.chunks; ++q) add(part[(int64_t)q * n + i]);
            double v = ((double)hi + (double)lo) * I.scale * inv;
            if (u) v = fma(-nrm, u[i], v);
            const int64_t vi = seg_base[sx] + (i - seg_i0[sx]);
            if (RBF_IN_RANGE(vi, a.rmax)) vs[vi] = v;
            bout[i] = qr[i] * inv;
        }
    }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        // dot partials: (segment, m) pairs
        for (int sx = 0; sx < nseg; ++sx) {
            if (!seg_act[sx]) continue;
            const int b = seg_b[sx];
            const BInst I = a.inst[b];
            const double* Q = a.side == 0 ? a.Z_all + (size_t)L * I.off : a.W_all + (size_t)(L + 1) * I.off;
            const int64_t i0 = seg_i0[sx];
            const int rows = (int)(seg_i1[sx] - i0);
            const int cslot = blockIdx.x - I.cfirst;
            const double* v = vs + seg_base[sx];
            // one warp per group of DG basis vectors, lanes along the rows
            // (coalesced loads of the basis columns); the DG lane sums are
            // reduced together by a transposing butterfly (offsets 16, 8, 4
            // halve the vectors a lane holds, the smaller offsets finish): 6 FP64
            // adds per lane for DG = 4 vectors instead of 5 per vector (8 vectors
            // per warp spilled registers at 4 CTAs per SM and were slower)
            for (int m0 = warp * DG; m0 < M; m0 += HB_WARPS * DG) {
                const int gc = min(DG, M - m0);
                double acc[DG];
#pragma unroll
                for (int g = 0; g < DG; ++g) acc[g] = 0.0;
                const double* q = Q + (int64_t)m0 * I.n + i0;
                for (int i = lane; i < rows; i += 32) {
                    const double vi = v[i];
#pragma unroll
                    for (int g = 0; g < DG; ++g)
                        if (g < gc) acc[g] = fma(q[(int64_t)g * I.n + i], vi, acc[g]);
                }
#pragma unroll
                for (int w = DG / 2, off = 16; w >= 1; w >>= 1, off >>= 1) {
                    const bool hi = (lane & off) != 0;
#pragma unroll
                    for (int g = 0; g < w; ++g) {
                        const double send = hi ? acc[g] : acc[g + w];
                        const double keep = hi ? acc[g + w] : acc[g];
                        acc[g] = keep + __shfl_xor_sync(RBF_FULL_MASK, send, off);
                    }
                }
                double t = acc[0];
#pragma unroll
                for (int off = 16 >> DG_LOG; off >= 1; off >>= 1) t += __shfl_xor_sync(RBF_FULL_MASK, t, off);
                const int m = m0 + ((lane >> (5 - DG_LOG)) & (DG - 1));  // the vector lane holds
                if ((lane & ((32 >> DG_LOG) - 1)) == 0 && m < M && RBF_IN_RANGE(cslot, I.ncta) &&
                    RBF_IN_RANGE(m, L + 2))
                    a.hpart_all[I.hoff + (int64_t)m * I.ncta + cslot] = t;
            }
        }
        if (!grid_sync_b(a.stt, a.bar, a.bar_group, a.budget)) return;
        // distributed reduction over all (instance, m) pairs
        {
            const int64_t P = (int64_t)a.B * M;
            for (int64_t p = (int64_t)blockIdx.x * HB_THREADS + threadIdx.x; p < P; p += (int64_t)G * HB_THREADS) {
                const int b = (int)(p / M), m = (int)(p % M);
                if (a.done_in[b]) continue;
                const BInst I = a.inst[b];
                const double* hp = a.hpart_all + I.hoff + (int64_t)m * I.ncta;
                double acc = 0.0;
                for (int s = 0; s < I.ncta; ++s) acc += __ldcg(hp + s);
                a.h_all[(size_t)b * (L + 2) + m] = acc;
            }
        }
        if (!grid_sync_b(a.stt, a.bar, a.bar_group, a.budget)) return;
        for (int sx = 0; sx < nseg; ++sx)
            for (int m = threadIdx.x; m < M; m += HB_THREADS)
                hs[sx * (L + 2) + m] = __ldcg(a.h_all + (size_t)seg_b[sx] * (L + 2) + m);
        __syncthreads();
        // v -= Q h over the slab rows: thread (row, group of basis vectors)
        const int row = threadIdx.x % UPD_ROWS_B;
        const int grp = threadIdx.x / UPD_ROWS_B;
        for (int base = 0; base < nrows; base += UPD_ROWS_B) {
            const int r = base + row;
            double c0 = 0.0, c1 = 0.0;
            int sx = 0;
            if (r < nrows) {
                while (sx + 1 < nseg && r >= seg_base[sx + 1]) ++sx;
                if (seg_act[sx]) {
                    const BInst I = a.inst[seg_b[sx]];
                    const double* Q = a.side == 0 ? a.Z_all + (size_t)L * I.off : a.W_all + (size_t)(L + 1) * I.off;
                    const double* q = Q + seg_i0[sx] + (r - seg_base[sx]);
                    const double* hh = hs + sx * (L + 2);
                    int m = grp;
                    for (; m + UPD_GROUPS_B < M; m += 2 * UPD_GROUPS_B) {
                        c0 = fma(q[(int64_t)m * I.n], hh[m], c0);
                        c1 = fma(q[(int64_t)(m + UPD_GROUPS_B) * I.n], hh[m + UPD_GROUPS_B], c1);
                    }
                    for (; m < M; m += UPD_GROUPS_B) c0 = fma(q[(int64_t)m * I.n], hh[m], c0);
                }
            }
            red[grp * UPD_ROWS_B + row] = c0 + c1;
            __syncthreads();
            if (grp == 0 && r < nrows && seg_act[sx]) {
                double t = 0.0;
#pragma unroll
                for (int gq = 0; gq < UPD_GROUPS_B; ++gq) t += red[gq * UPD_ROWS_B + row];
                vs[r] -= t;
            }
            __syncthreads();
        }
    }
    // ---- store v (+ FP32 copy) and the per-instance |v|^2 partials of this slab
    for (int sx = 0; sx < nseg; ++sx) {
        if (!seg_act[sx]) continue;  // uniform across the CTA
        const BInst I = a.inst[seg_b[sx]];
        const int rows = (int)(seg_i1[sx] - seg_i0[sx]);
        double acc = 0.0;
        for (int i = threadIdx.x; i < rows; i += HB_THREADS) {
            const double t = vs[seg_base[sx] + i];
            a.v_all[I.off + seg_i0[sx] + i] = t;
            a.v32_all[I.off + seg_i0[sx] + i] = (float)t;
            acc = fma(t, t, acc);
        }
        acc = warp_sum(acc);
        __syncthreads();
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < HB_WARPS; ++w) t += red[w];
            a.npart_all[I.noff + (blockIdx.x - I.cfirst)] = t;
        }
        __syncthreads();
    }
}

// Start of the run: per-instance |f|^2 partials over the half-step slabs, copy
// of f into q_raw (FP64 and FP32), per-instance state reset.
__global__ void __launch_bounds__(HB_THREADS) k_init_batch(HalfBArgs a, const double* __restrict__ f_all,
                                                           double* __restrict__ q_all) {
    __shared__ double red[HB_WARPS];
    const int G = gridDim.x;
    const int64_t R0 = a.T * blockIdx.x / G, R1 = a.T * (blockIdx.x + 1) / G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int b = 0;
    while (b + 1 < a.B && a.offs[b + 1] <= R0) ++b;
    for (; b < a.B && a.offs[b] < R1; ++b) {
        const BInst I = a.inst[b];
        const int64_t g0 = max(R0, a.offs[b]), g1 = min(R1, a.offs[b + 1]);
        if (g1 <= g0) continue;
        double acc = 0.0;
        for (int64_t g = g0 + threadIdx.x; g < g1; g += HB_THREADS) {
            const double t = f_all[g];
            q_all[g] = t;
            a.v32_all[g] = (float)t;
            acc = fma(t, t, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < HB_WARPS; ++w) t += red[w];
            a.npart_all[I.noff + (blockIdx.x - I.cfirst)] = t;
            if ((int)blockIdx.x == I.cfirst) {
                a.chat_all[2 * b] = a.chat_all[2 * b + 1] = 0.0;
                a.binfo[BI_STEPS * a.B + b] = 0;
                a.binfo[BI_BREAK * a.B + b] = 0;
                a.binfo[BI_DONE0 * a.B + b] = 0;
                a.binfo[BI_DONE1 * a.B + b] = 0;
            }
        }
        __syncthreads();
    }
}

// beta_{l+1} and w_{l+1} per instance (one block per instance).
__global__ void k_final_batch(HalfBArgs a, int l) {
    __shared__ double red[32];
    __shared__ double inv_s;
    __shared__ int brk_s;
    const int b = blockIdx.x;
    if (a.done_in[b]) return;
    const BInst I = a.inst[b];
    double acc = 0.0;
    for (int q = threadIdx.x; q < I.ncta; q += blockDim.x) acc += a.npart_all[I.noff + q];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double nrm = sqrt(t);
        double* ch = a.chat_all + 2 * b;
        const double chn = fmax(ch[(l + 1) & 1], hypot(a.alpha_all[(size_t)b * a.L + l - 1], nrm));
        const bool nonfinite = !isfinite(nrm);
        if (!nonfinite) ch[0] = ch[1] = chn;
        const int brk = (nrm <= a.factor * (double)I.n * DBL_EPSILON * chn || nonfinite) ? 2 : 0;
        a.beta_all[(size_t)b * (a.L + 1) + l] = brk ? 0.0 : nrm;
        a.binfo[BI_STEPS * a.B + b] = l;
        a.binfo[BI_BREAK * a.B + b] = nonfinite ? 3 : brk;
        inv_s = 1.0 / nrm;
        brk_s = brk;
    }
    __syncthreads();
    double* w = a.W_all + (size_t)(a.L + 1) * I.off + (int64_t)l * I.n;
    const double* q = a.qraw_all + I.off;
    for (int64_t i = threadIdx.x; i < I.n; i += blockDim.x) w[i] = brk_s ? 0.0 : q[i] * inv_s;
}

// ---------------------------------------------------------------------------
// Autotuner candidates for the batched product.
// ---------------------------------------------------------------------------
struct MfCand {
    int ro, th;  // rows per lane (blocks of 32 ro nodes), threads per CTA
};
constexpr MfCand MF_CANDS[] = {{4, MS_W * 32}, {8, MS_W * 32}};
constexpr int N_CANDS = sizeof(MF_CANDS) / sizeof(MF_CANDS[0]);

template <int TRANS>
void launch_mf_cand(int c, int items, cudaStream_t s, const MfItem* it, const BInst* in, const float* X32,
                    const float* x32, float* part, const int* done) {
    if (c == 0) k_mf_batch<TRANS, 4><<<items, MS_W * 32, 0, s>>>(it, in, X32, x32, part, done);
    else k_mf_batch<TRANS, 8><<<items, MS_W * 32, 0, s>>>(it, in, X32, x32, part, done);
}

// Host-side description of one batch shape and its device tables.
struct BatchPlan {
    int B = 0, L = 0, G = 0, rmax = 0, bar_group = 0, bar_k = 0;
    int64_t T = 0;
    std::vector<BInst> inst;
    std::vector<int64_t> offs;
    int64_t part_total = 0, part_max = 0, hpart_total = 0;
    int npart_total = 0;
};

}  // namespace

// Tuning and graph state lives in the context (one entry; a new batch shape
// re-tunes and re-captures).
constexpr int GRAPH_SLOTS = 4;  // captured step loops kept per context (e.g. a short and a full run)

struct BatchTuneState {
    int64_t key_T = -1;
    int key_B = -1;
    int cand = 1;
    double best_ms = 0.0;
    int graph_kernels = 0;               // kernels in the graph used last
    cudaGraphExec_t exec[GRAPH_SLOTS] = {};
    std::vector<unsigned char> graph_key[GRAPH_SLOTS];  // exact bytes of what each graph bakes in
    int slot_kernels[GRAPH_SLOTS] = {};
    uint64_t last_use[GRAPH_SLOTS] = {};
    uint64_t clock = 0;
    cudaStream_t stream = nullptr;
    void drop_graphs() {
        for (int i = 0; i < GRAPH_SLOTS; ++i) {
            if (exec[i]) cudaGraphExecDestroy(exec[i]);
            exec[i] = nullptr;
            graph_key[i].clear();
        }
    }
};

static BatchTuneState& tune_state(rbf_ctx* ctx) {
    if (!ctx->batch_state) ctx->batch_state = new BatchTuneState();
    return *(BatchTuneState*)ctx->batch_state;
}

cudaStream_t rbf_batch_stream(rbf_ctx* ctx) {
    return ctx->batch_state ? ((BatchTuneState*)ctx->batch_state)->stream : nullptr;
}

void rbf_batch_state_free(rbf_ctx* ctx) {
    if (!ctx->batch_state) return;
    BatchTuneState* ts = (BatchTuneState*)ctx->batch_state;
    ts->drop_graphs();
    if (ts->stream) cudaStreamDestroy(ts->stream);
    delete ts;
    ctx->batch_state = nullptr;
}

// Blocks of 32 ro nodes per instance for the tile-pair product: one partial
// slot per block, instance after instance.
static void set_blocks(BatchPlan* P, int ro) {
    const int64_t Bk = 32 * (int64_t)ro;
    int64_t poff = 0;
    for (BInst& I : P->inst) {
        I.chunks = (int)((I.n + Bk - 1) / Bk);
        I.poff = poff;
        poff += (int64_t)I.chunks * I.n;
    }
    P->part_total = poff;
}

static rbf_status plan_batch(rbf_ctx* ctx, const rbf_batch* bt, int form, BatchPlan* P) {
    const int B = bt->count;
    P->B = B;
    P->L = bt->capacity;
    P->offs.assign(B + 1, 0);
    for (int b = 0; b < B; ++b) P->offs[b + 1] = P->offs[b] + bt->n[b];
    P->T = P->offs[B];
    // cooperative grid: up to 4 co-resident CTAs per SM (measured on the 96-instance
    // sweep: 0.663 ms per half-step against 0.691 with 8 and 0.728 with 2), at least 64 rows per
    // CTA; the shared memory depends on the slab size, so iterate to a fixed point
    cudaFuncSetAttribute(k_half_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int64_t G = (int64_t)ctx->sm_count * 4;
    for (int it = 0; it < 6; ++it) {
        if (G > P->T / 64) G = P->T / 64;
        if (G < 1) G = 1;
        const int64_t rmax = (P->T + G - 1) / G;
        const size_t smem = ((size_t)rmax + (size_t)SEGMAX * (P->L + 2)) * sizeof(double);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_half_batch, HB_THREADS, smem);
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 4) per_sm = 4;
        const int64_t G2 = std::min<int64_t>((int64_t)ctx->sm_count * per_sm, std::max<int64_t>(1, P->T / 64));
        if (G2 >= G) break;
        G = G2;
    }
    cudaGetLastError();
    P->G = (int)G;
    P->rmax = (int)((P->T + G - 1) / G);
    P->bar_group = 1;
    while (P->bar_group * P->bar_group < P->G) ++P->bar_group;
    P->bar_k = (P->G + P->bar_group - 1) / P->bar_group;
    P->inst.resize(B);
    int64_t poff = 0, hoff = 0;  // (partials: set_blocks)
    int noff = 0;
    for (int b = 0; b < B; ++b) {
        BInst& I = P->inst[b];
        I.off = P->offs[b];
        I.n = bt->n[b];
        I.ni = bt->n_interior[b];
        I.c2 = (float)(bt->c[b] * bt->c[b]);
        I.k2 = (float)(bt->k[b] * bt->k[b]);
        I.scale = form == RBF_FORM_EPS ? 1.0 / bt->c[b] : 1.0;
        // CTAs whose balanced slab [T c / G, T (c+1) / G) intersects [off, off+n)
        const int64_t r0 = I.off, r1 = I.off + I.n;
        int c0 = (int)((r0 * G) / P->T);
        while (c0 > 0 && (P->T * c0) / G > r0) --c0;
        while (c0 + 1 < G && (P->T * (c0 + 1)) / G <= r0) ++c0;
        int c1 = (int)(((r1 - 1) * G) / P->T);
        while (c1 > 0 && (P->T * c1) / G > r1 - 1) --c1;
        while (c1 + 1 < G && (P->T * (c1 + 1)) / G <= r1 - 1) ++c1;
        I.cfirst = c0;
        I.ncta = c1 - c0 + 1;
        I.hoff = hoff;
        hoff += (int64_t)(P->L + 2) * I.ncta;
        I.noff = noff;
        noff += I.ncta;
    }
    (void)poff;
    set_blocks(P, MF_CANDS[0].ro);  // the smallest blocks: the most partial slots, for the workspace
    P->part_max = P->part_total;
    P->hpart_total = hoff;
    P->npart_total = noff;
    // segment bound: a slab must meet at most SEGMAX instances
    for (int c = 0; c < P->G; ++c) {
        const int64_t R0 = P->T * c / G, R1 = P->T * (c + 1) / G;
        int cnt = 0;
        for (int b = 0; b < B; ++b)
            if (P->offs[b] < R1 && P->offs[b + 1] > R0) ++cnt;
        if (cnt > SEGMAX)
            return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "a row slab meets %d instances (max %d): instances too small", cnt,
                            SEGMAX);
    }
    return RBF_OK;
}

// Every tile (bi <= bj) of every instance for blocks of 32 ro nodes, largest
// instances first (longest-processing-time order for the block scheduler).
static std::vector<MfItem> make_items(const BatchPlan& P, int ro) {
    const int64_t Bk = 32 * (int64_t)ro;
    std::vector<int> order(P.B);
    for (int b = 0; b < P.B; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return P.inst[x].n > P.inst[y].n; });
    std::vector<MfItem> items;
    for (int b : order) {
        const int nb = (int)((P.inst[b].n + Bk - 1) / Bk);
        for (int i = 0; i < nb; ++i)
            for (int j = i; j < nb; ++j) items.push_back({b, i, j});
    }
    return items;
}

extern "C" rbf_status rbf_get_tuning(const rbf_ctx* ctx, rbf_tuning* out) {
    if (!ctx || !out) return RBF_ERR_INVALID;
    BatchTuneState& ts = tune_state(const_cast<rbf_ctx*>(ctx));
    out->mf_outputs_per_thread = MF_CANDS[ts.cand].ro;
    out->mf_threads = MF_CANDS[ts.cand].th;
    out->candidates = N_CANDS;
    out->best_ms = ts.best_ms;
    out->graph_kernels = ts.graph_kernels;
    return RBF_OK;
}

namespace {

struct BatchWs {
    BInst* inst;
    int64_t* offs;
    MfItem* items;
    float* part;  // the products' partial slots (FP32 runs, unscaled)
    float* X32;  // node coordinates rounded to FP32, like the nodes [3][n] per instance
    double* hpart;
    double* h;
    double* npart;
    double* vr;
    double* vp;
    float* vr32;
    float* vp32;
    int* binfo;
    double* chat;
    unsigned* bar;
    size_t bytes;
};

size_t batch_ws_layout(const BatchPlan& P, size_t n_items_max, BatchWs* w, void* base) {
    WsCarve wc(base ? base : (void*)0x100);  // dry run when base is null
    BatchWs t;
    t.inst = wc.take<BInst>(P.B);
    t.offs = wc.take<int64_t>(P.B + 1);
    t.items = wc.take<MfItem>(n_items_max);
    t.part = wc.take<float>(P.part_max);
    t.X32 = wc.take<float>((size_t)3 * P.T);
    t.hpart = wc.take<double>(P.hpart_total);
    t.h = wc.take<double>((size_t)P.B * (P.L + 2));
    t.npart = wc.take<double>(P.npart_total);
    t.vr = wc.take<double>(P.T);
    t.vp = wc.take<double>(P.T);
    t.vr32 = wc.take<float>(P.T);
    t.vp32 = wc.take<float>(P.T);
    t.binfo = wc.take<int>((size_t)6 * P.B);
    t.chat = wc.take<double>((size_t)2 * P.B);
    t.bar = wc.take<unsigned>((size_t)(P.bar_k + 2) * BAR_STRIDE_B);
    t.bytes = wc.off + 256;
    if (w) *w = t;
    return t.bytes;
}

size_t max_items(const BatchPlan& P) {
    size_t m = 0;
    for (int c = 0; c < N_CANDS; ++c) {
        const int64_t Bk = 32 * (int64_t)MF_CANDS[c].ro;
        size_t cnt = 0;
        for (int b = 0; b < P.B; ++b) {
            const size_t nb = (size_t)((P.inst[b].n + Bk - 1) / Bk);
            cnt += nb * (nb + 1) / 2;
        }
        if (cnt > m) m = cnt;
    }
    return m;
}

}  // namespace

extern "C" rbf_status rbf_batch_gkb(rbf_ctx* ctx, rbf_batch* bt, int steps, int form) {
    RbfRange range_("rbf_batch_gkb");
    if (!ctx) return RBF_ERR_INVALID;
    if (!bt || bt->count < 1 || !bt->n || !bt->n_interior || !bt->c || !bt->k || !bt->d_nodes || !bt->d_f ||
        !bt->d_W || !bt->d_Z || !bt->d_alpha || !bt->d_beta || !bt->steps_done || !bt->breakdown)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_batch_gkb: missing field");
    if (steps < 1 || steps > bt->capacity || bt->capacity > 1022)
        return rbf_fail(ctx, RBF_ERR_INVALID, "steps %d outside [1, capacity %d] (capacity <= 1022)", steps,
                        bt->capacity);
    if (form != RBF_FORM_C && form != RBF_FORM_EPS) return rbf_fail(ctx, RBF_ERR_INVALID, "unknown form");
    for (int b = 0; b < bt->count; ++b) {
        if (bt->n[b] < 1 || bt->n_interior[b] < 0 || bt->n_interior[b] > bt->n[b] || !(bt->c[b] > 0) ||
            !(bt->k[b] >= 0))
            return rbf_fail(ctx, RBF_ERR_INVALID, "instance %d: invalid n, n_interior, c or k", b);
        if (steps > bt->n[b]) return rbf_fail(ctx, RBF_ERR_INVALID, "instance %d: steps exceed n", b);
        if (bt->steps_limit && bt->steps_limit[b] < 1)
            return rbf_fail(ctx, RBF_ERR_INVALID, "instance %d: steps_limit must be >= 1", b);
    }
    BatchPlan P;
    RBF_TRY(plan_batch(ctx, bt, form, &P));
    if (P.rmax + SEGMAX * (P.L + 2) > 24 * 1024)
        return rbf_fail(ctx, RBF_ERR_UNSUPPORTED, "batch slab too large for shared memory");
    const size_t nitems = max_items(P);
    RBF_TRY(rbf_ws_reserve(ctx, batch_ws_layout(P, nitems, nullptr, nullptr)));
    BatchWs w;
    batch_ws_layout(P, nitems, &w, ctx->ws);
    BatchTuneState& ts = tune_state(ctx);
    if (!ts.stream) RBF_CUDA(ctx, cudaStreamCreateWithFlags(&ts.stream, cudaStreamNonBlocking));
    cudaStream_t s = ts.stream;
    // order the batch work after the context stream's earlier work
    RBF_CUDA(ctx, cudaEventRecord(ctx->ev[0], ctx->stream));
    RBF_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev[0], 0));
    RBF_CUDA(ctx, cudaMemcpyAsync(w.inst, P.inst.data(), sizeof(BInst) * P.B, cudaMemcpyHostToDevice, s));
    RBF_CUDA(ctx, cudaMemcpyAsync(w.offs, P.offs.data(), sizeof(int64_t) * (P.B + 1), cudaMemcpyHostToDevice, s));
    RBF_CUDA(ctx, cudaMemsetAsync(w.bar, 0, (size_t)(P.bar_k + 2) * BAR_STRIDE_B * sizeof(unsigned), s));
    RBF_CUDA(ctx, cudaMemsetAsync(w.binfo, 0, sizeof(int) * 6 * P.B, s));
    std::vector<int> lim((size_t)P.B, steps);
    if (bt->steps_limit)
        for (int b = 0; b < P.B; ++b) lim[b] = bt->steps_limit[b] < steps ? bt->steps_limit[b] : steps;
    RBF_CUDA(ctx, cudaMemcpyAsync(w.binfo + BI_LIMIT * P.B, lim.data(), sizeof(int) * P.B, cudaMemcpyHostToDevice, s));
    rbf_dev_state* dst = ctx->d_state;
    RBF_CUDA(ctx, cudaMemsetAsync(&dst->info[IN_ERR], 0, sizeof(int), s));

    HalfBArgs a{};
    a.inst = w.inst;
    a.offs = w.offs;
    a.B = P.B;
    a.T = P.T;
    a.L = P.L;
    a.factor = ctx->opt.breakdown_factor;
    a.alpha_all = bt->d_alpha;
    a.beta_all = bt->d_beta;
    a.W_all = bt->d_W;
    a.Z_all = bt->d_Z;
    a.part_all = w.part;
    a.hpart_all = w.hpart;
    a.h_all = w.h;
    a.npart_all = w.npart;
    a.binfo = w.binfo;
    a.chat_all = w.chat;
    a.stt = dst;
    a.bar = w.bar;
    a.bar_group = P.bar_group;
    a.budget = ctx->opt.wait_budget;
    a.rmax = P.rmax;
    a.qraw_all = w.vp;
    a.v32_all = w.vp32;
    a.done_in = w.binfo + BI_DONE0 * P.B;
    a.limit = w.binfo + BI_LIMIT * P.B;
    k_init_batch<<<P.G, HB_THREADS, 0, s>>>(a, bt->d_f, w.vp);
    RBF_LAUNCHED(ctx, "k_init_batch");
    RBF_TRY(launch_to_f32(ctx, 3 * P.T, bt->d_nodes, w.X32, s));  // the products' FP32 node coordinates

    // ---- autotune the product tile on this batch (first time this shape is seen)
    if (ts.key_T != P.T || ts.key_B != P.B) {
        cudaEvent_t e0, e1;
        RBF_CUDA(ctx, cudaEventCreate(&e0));
        RBF_CUDA(ctx, cudaEventCreate(&e1));
        double best = 1e30;
        int bestc = 1;
        for (int c = 0; c < N_CANDS; ++c) {
            set_blocks(&P, MF_CANDS[c].ro);
            std::vector<MfItem> items = make_items(P, MF_CANDS[c].ro);
            RBF_CUDA(ctx, cudaMemcpyAsync(w.inst, P.inst.data(), sizeof(BInst) * P.B, cudaMemcpyHostToDevice, s));
            RBF_CUDA(ctx, cudaMemcpyAsync(w.items, items.data(), sizeof(MfItem) * items.size(),
                                          cudaMemcpyHostToDevice, s));
            float ms_sum = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                RBF_CUDA(ctx, cudaEventRecord(e0, s));
                launch_mf_cand<1>(c, (int)items.size(), s, w.items, w.inst, w.X32, w.vp32, w.part, nullptr);
                launch_mf_cand<0>(c, (int)items.size(), s, w.items, w.inst, w.X32, w.vp32, w.part, nullptr);
                RBF_CUDA(ctx, cudaEventRecord(e1, s));
                RBF_CUDA(ctx, cudaEventSynchronize(e1));
                float ms = 0.f;
                RBF_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
                if (rep == 1) ms_sum = ms;  // second run: warm
                ctx->launches += 2;
            }
            if (ms_sum < best) {
                best = ms_sum;
                bestc = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ts.key_T = P.T;
        ts.key_B = P.B;
        ts.cand = bestc;
        ts.best_ms = best;
        ts.drop_graphs();
    }
    const int cand = ts.cand;
    set_blocks(&P, MF_CANDS[cand].ro);
    std::vector<MfItem> items = make_items(P, MF_CANDS[cand].ro);
    RBF_CUDA(ctx, cudaMemcpyAsync(w.inst, P.inst.data(), sizeof(BInst) * P.B, cudaMemcpyHostToDevice, s));
    RBF_CUDA(ctx, cudaMemcpyAsync(w.items, items.data(), sizeof(MfItem) * items.size(), cudaMemcpyHostToDevice, s));
    const int nit = (int)items.size();
    const size_t hsmem = ((size_t)P.rmax + (size_t)SEGMAX * (P.L + 2)) * sizeof(double);
    if (hsmem > 48 * 1024)
        RBF_CUDA(ctx, cudaFuncSetAttribute(k_half_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem));

    // ---- the step loop, captured into one graph.  A cached graph is reused only
    // when every value it bakes in is the same, compared byte for byte: the
    // half-step arguments (all pointers, sizes and the budget), the product's
    // grid (item count, tile candidate), the workspace slices the launches
    // read and write, the node and input pointers, the cooperative grid, its
    // shared memory and the step count.
    std::vector<unsigned char> key;
    auto put = [&key](const auto& v) {
        const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
        key.insert(key.end(), b, b + sizeof(v));
    };
    put(a.inst); put(a.offs); put(a.B); put(a.T); put(a.L); put(a.factor);
    put(a.alpha_all); put(a.beta_all); put(a.W_all); put(a.Z_all); put(a.part_all); put(a.hpart_all);
    put(a.h_all); put(a.npart_all); put(a.binfo); put(a.limit); put(a.chat_all); put(a.stt); put(a.bar);
    put(a.bar_group); put(a.budget); put(a.rmax);
    put(bt->d_nodes); put(bt->d_f); put(w.items); put(w.part); put(w.X32); put(w.vr); put(w.vp); put(w.vr32); put(w.vp32);
    put(nit); put(cand); put(P.G); put(hsmem); put(steps); put(form); put(s);
    // per-launch timing (opt.timing bit 1): the loop is launched directly, each
    // launch between CUDA events on the batch stream
    const bool timed = (ctx->opt.timing & 2) != 0;
    auto record_steps = [&](int* kernels) -> cudaError_t {
        int cnt = 0;
        for (int j = 1; j <= steps; ++j) {
            for (int side = 0; side < 2; ++side) {
                const int half = 2 * (j - 1) + side;  // launch index: done flags alternate
                const int* din = w.binfo + (half & 1 ? BI_DONE1 : BI_DONE0) * P.B;
                int* dout = w.binfo + (half & 1 ? BI_DONE0 : BI_DONE1) * P.B;
                const int trans = side == 0 ? 1 : 0;
                const float* x32 = side == 0 ? w.vp32 : w.vr32;
                const int pslot = timed ? rbf_prod_begin(ctx, trans, s) : -1;
                if (trans)
                    launch_mf_cand<1>(cand, nit, s, w.items, w.inst, w.X32, x32, w.part, din);
                else
                    launch_mf_cand<0>(cand, nit, s, w.items, w.inst, w.X32, x32, w.part, din);
                rbf_prod_end(ctx, trans, pslot, s);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) return e;
                HalfBArgs h = a;
                h.j = j;
                h.side = side;
                h.qraw_all = side == 0 ? w.vp : w.vr;
                h.v_all = side == 0 ? w.vr : w.vp;
                h.v32_all = side == 0 ? w.vr32 : w.vp32;
                h.done_in = din;
                h.done_out = dout;
                void* args[] = {&h};
                const int rslot = timed ? rbf_prod_begin(ctx, 2, s) : -1;
                e = cudaLaunchCooperativeKernel((const void*)k_half_batch, dim3(P.G), dim3(HB_THREADS), args, hsmem, s);
                rbf_prod_end(ctx, 2, rslot, s);
                if (e != cudaSuccess) return e;
                cnt += 2;
            }
        }
        if (kernels) *kernels = cnt;
        return cudaSuccess;
    };
    bool ran = false;
    int slot = -1;
    for (int i = 0; i < GRAPH_SLOTS; ++i)
        if (ts.exec[i] && ts.graph_key[i] == key) slot = i;
    if (timed) {
        ts.graph_kernels = 0;  // launched directly below
    } else if (slot >= 0) {
        ts.last_use[slot] = ++ts.clock;
        ts.graph_kernels = ts.slot_kernels[slot];
        RBF_CUDA(ctx, cudaGraphLaunch(ts.exec[slot], s));
        ran = true;
    } else {
        slot = 0;  // an empty slot, else the least recently used one
        for (int i = 0; i < GRAPH_SLOTS; ++i) {
            if (!ts.exec[i]) {
                slot = i;
                break;
            }
            if (ts.last_use[i] < ts.last_use[slot]) slot = i;
        }
        if (ts.exec[slot]) {
            cudaGraphExecDestroy(ts.exec[slot]);
            ts.exec[slot] = nullptr;
        }
        cudaGraph_t graph = nullptr;
        int kernels = 0;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t er = record_steps(&kernels);
            e = cudaStreamEndCapture(s, &graph);
            if (er != cudaSuccess) e = er;
        }
        if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&ts.exec[slot], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess && ts.exec[slot]) {
            ts.graph_key[slot] = key;  // a copy
            ts.slot_kernels[slot] = kernels;
            ts.last_use[slot] = ++ts.clock;
            ts.graph_kernels = kernels;
            RBF_CUDA(ctx, cudaGraphLaunch(ts.exec[slot], s));
            ran = true;
        } else {
            cudaGetLastError();  // capture unsupported: launch the same sequence directly
            ts.exec[slot] = nullptr;
            ts.graph_kernels = 0;
        }
    }
    if (!ran) {
        cudaError_t e = record_steps(nullptr);
        if (e != cudaSuccess)
            return rbf_fail(ctx, RBF_ERR_CUDA, "batched GKB launch failed: %s", cudaGetErrorString(e));
    }
    ctx->launches += 4LL * steps;
    // beta_{l+1}, w_{l+1}
    {
        const int last = 2 * steps;  // launch index after the loop
        HalfBArgs h = a;
        h.qraw_all = w.vp;
        h.done_in = w.binfo + (last & 1 ? BI_DONE1 : BI_DONE0) * P.B;
        k_final_batch<<<P.B, 256, 0, s>>>(h, steps);
        RBF_LAUNCHED(ctx, "k_final_batch");
    }
    // results back to the host
    std::vector<int> info(6 * (size_t)P.B);
    RBF_CUDA(ctx, cudaMemcpyAsync(info.data(), w.binfo, sizeof(int) * 6 * P.B, cudaMemcpyDeviceToHost, s));
    int err = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&err, &dst->info[IN_ERR], sizeof(int), cudaMemcpyDeviceToHost, s));
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    RBF_CUDA(ctx, cudaGetLastError());
    RBF_TRY(rbf_check_all(ctx));
    for (int b = 0; b < P.B; ++b) {
        bt->steps_done[b] = info[BI_STEPS * P.B + b];
        bt->breakdown[b] = info[BI_BREAK * P.B + b];
    }
    // steps_done as a device array for the projected phase (first row of binfo)
    if (err) return rbf_fail(ctx, (rbf_status)err, "a bounded grid barrier of the batched GKB gave up");
    return RBF_OK;
}

static rbf_status batch_hkt_impl(rbf_ctx* ctx, const rbf_batch* bt, int rule, const int* h_rules,
                                 const double* h_lambda_in, double* d_coef, double* h_lambda) {
    const int B = bt->count, L = bt->capacity;
    int lmax = 0;
    for (int b = 0; b < B; ++b) lmax = bt->steps_done[b] > lmax ? bt->steps_done[b] : lmax;
    if (lmax < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "no instance has a completed step");
    std::vector<int64_t> tab(3 * (size_t)B);
    int64_t off = 0, nmax = 0;
    for (int b = 0; b < B; ++b) {
        tab[b] = bt->n[b];
        tab[B + b] = (int64_t)L * off;  // Z_b offset
        tab[2 * B + b] = off;           // coef_b offset
        off += bt->n[b];
        nmax = bt->n[b] > nmax ? bt->n[b] : nmax;
    }
    const size_t extra = ws_align(sizeof(int64_t) * 3 * B) + ws_align(sizeof(int) * B) + ws_align(sizeof(double) * B) +
                         ws_align(sizeof(int) * B) + ws_align(sizeof(int) * B) + ws_align(sizeof(double) * B);
    RBF_TRY(rbf_ws_reserve(ctx, extra + select_ws_bytes_batch(ctx, L, B)));
    WsCarve wc(ctx->ws);
    int64_t* dtab = wc.take<int64_t>(3 * (size_t)B);
    int* l_arr = wc.take<int>(B);
    double* lam = wc.take<double>(B);
    int* idx = wc.take<int>(B);
    int* rules = wc.take<int>(B);
    double* lam_in = wc.take<double>(B);
    void* rest = (void*)wc.take<char>(select_ws_bytes_batch(ctx, L, B));
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaMemcpyAsync(dtab, tab.data(), sizeof(int64_t) * 3 * B, cudaMemcpyHostToDevice, s));
    RBF_CUDA(ctx, cudaMemcpyAsync(l_arr, bt->steps_done, sizeof(int) * B, cudaMemcpyHostToDevice, s));
    if (h_rules) {
        RBF_CUDA(ctx, cudaMemcpyAsync(rules, h_rules, sizeof(int) * B, cudaMemcpyHostToDevice, s));
        RBF_CUDA(ctx, cudaMemcpyAsync(lam_in, h_lambda_in, sizeof(double) * B, cudaMemcpyHostToDevice, s));
    }
    ProjDims d{B, L, 0, l_arr};
    LiftDims ld{dtab, dtab + B, dtab + 2 * B, 0, 0, nmax};
    RBF_TRY(launch_select_batch(ctx, d, 0, rule, 0.0, 0, bt->d_alpha, bt->d_beta, bt->d_Z, ld, d_coef, nullptr, rest,
                                lam, idx, nullptr, false, h_rules ? rules : nullptr, h_rules ? lam_in : nullptr));
    RBF_CUDA(ctx, cudaMemcpyAsync(h_lambda, lam, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    RBF_CUDA(ctx, cudaGetLastError());
    return RBF_OK;
}

extern "C" rbf_status rbf_batch_hkt(rbf_ctx* ctx, const rbf_batch* bt, int rule, double* d_coef, double* h_lambda) {
    RbfRange range_("rbf_batch_hkt");
    if (!ctx) return RBF_ERR_INVALID;
    if (!bt || !d_coef || !h_lambda || bt->count < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_batch_hkt: NULL argument");
    if (rule != RBF_GCV && rule != RBF_LCURVE) return rbf_fail(ctx, RBF_ERR_INVALID, "rule must be GCV or L-curve");
    return batch_hkt_impl(ctx, bt, rule, nullptr, nullptr, d_coef, h_lambda);
}

extern "C" rbf_status rbf_batch_hkt_each(rbf_ctx* ctx, const rbf_batch* bt, const int* h_rules,
                                         const double* h_lambda_in, double* d_coef, double* h_lambda) {
    RbfRange range_("rbf_batch_hkt_each");
    if (!ctx) return RBF_ERR_INVALID;
    if (!bt || !h_rules || !h_lambda_in || !d_coef || !h_lambda || bt->count < 1)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_batch_hkt_each: NULL argument");
    for (int b = 0; b < bt->count; ++b) {
        const int r = h_rules[b];
        if (r != RBF_GCV && r != RBF_LCURVE && r != RBF_FIXED && r != RBF_FIXED_T)
            return rbf_fail(ctx, RBF_ERR_INVALID, "instance %d: unknown rule %d", b, r);
        if (r == RBF_FIXED && !(h_lambda_in[b] >= 0.0))
            return rbf_fail(ctx, RBF_ERR_INVALID, "instance %d: fixed lambda must be >= 0", b);
        if (r == RBF_FIXED_T && !(h_lambda_in[b] >= -300.0 && h_lambda_in[b] <= 300.0))
            return rbf_fail(ctx, RBF_ERR_INVALID, "instance %d: fixed t must be finite", b);
    }
    return batch_hkt_impl(ctx, bt, RBF_GCV, h_rules, h_lambda_in, d_coef, h_lambda);
}

extern "C" rbf_status rbf_batch_evaluate(rbf_ctx* ctx, const rbf_batch* bt, int form, const double* d_coef,
                                         const double* d_points, const int64_t* m, double* d_u) {
    RbfRange range_("rbf_batch_evaluate");
    if (!ctx) return RBF_ERR_INVALID;
    if (!bt || !d_coef || !d_points || !m || !d_u) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_batch_evaluate: NULL");
    int64_t off = 0, moff = 0;
    for (int b = 0; b < bt->count; ++b) {
        rbf_operator op{};
        op.d_nodes = bt->d_nodes + 3 * off;
        op.n = bt->n[b];
        op.n_interior = bt->n_interior[b];
        op.c = bt->c[b];
        op.k = bt->k[b];
        op.storage = RBF_MATRIX_FREE;
        op.precision = RBF_MIXED;
        op.form = form;
        if (m[b] > 0) RBF_TRY(launch_evaluate(ctx, &op, d_coef + off, d_points + 3 * moff, m[b], d_u + moff));
        off += bt->n[b];
        moff += m[b];
    }
    return RBF_OK;
}

RBF_CHECK_READER(batch)
