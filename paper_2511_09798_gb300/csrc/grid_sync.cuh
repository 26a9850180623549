// Bounded two-level grid barrier for cooperative kernels (one CTA per slot of
// a cooperative launch).
#pragma once

#include "common.cuh"
#include "internal.h"

// ---------------------------------------------------------------------------
// Grid barrier for cooperative kernels: two levels so that no
// L2 address sees more than ~sqrt(G) atomics (one address with all G CTAs
// serialises ~14 ns per atomic).  bar[0..K) are group counters, bar[K] the top
// counter, bar[K+1] the generation; each on its own 128-byte line (stride 32).
// Bounded: after `budget` polls it records RBF_ERR_TIMEOUT in the device state,
// stops the run and returns false; the caller's CTA then exits without further
// barriers.
// ---------------------------------------------------------------------------
static constexpr int BAR_STRIDE = 32;

static __device__ bool grid_sync(rbf_dev_state* __restrict__ stt, unsigned* __restrict__ bar, int group,
                                 long long budget) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int G = gridDim.x;
        const int K = (G + group - 1) / group;
        const int grp = blockIdx.x / group;
        const int members = min(group, G - grp * group);
        unsigned* sub = bar + (size_t)grp * BAR_STRIDE;
        unsigned* top = bar + (size_t)K * BAR_STRIDE;
        volatile unsigned* gen = bar + (size_t)(K + 1) * BAR_STRIDE;
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
                atomicExch(&stt->info[IN_DONE], 1);
                break;
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}


// ---------------------------------------------------------------------------
// Grid barrier number `epoch` (1, 2, ... since the counters were zeroed) that
// also reduces per-CTA partial sums.  part is [M][G] (CTA b wrote
// part[m * G + b]); on a true return every CTA holds in hs (shared memory)
//   hs[m] = sum over groups q = 0..K-1 of ( sum over the CTAs b of group q of
//           part[m * G + b] ),
// each sum taken in a fixed order (two interleaved chains, then their sum),
// so the result does not depend on which CTA arrives last.  The counters only
// grow: the last CTA to arrive in a group (its counter reaches
// members * epoch) sums the group's columns into gpart (two buffers by epoch
// parity, so that a slow CTA still reading the previous sums is never
// overwritten) and then adds 1 to the top counter with release semantics;
// every CTA waits (acquire) for the top counter to reach K * epoch and sums
// the K group sums itself.  With M = 0 it is a plain barrier.  Bounded: after
// `budget` polls it records RBF_ERR_TIMEOUT, stops the run and returns false.
// ---------------------------------------------------------------------------
static __device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
static __device__ __forceinline__ void red_add_release_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
static __device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

static __device__ bool grid_reduce_sync(rbf_dev_state* __restrict__ stt, unsigned* __restrict__ bar, int group,
                                        long long budget, unsigned epoch, const double* __restrict__ part,
                                        double* __restrict__ gpart, double* __restrict__ hs, int M,
                                        int64_t gpart_len) {
    __shared__ int role;
    __shared__ int ok;
    const int G = gridDim.x;
    const int K = (G + group - 1) / group;
    const int grp = blockIdx.x / group;
    const int b0 = grp * group;
    const int members = min(group, G - b0);
    unsigned* sub = bar + (size_t)grp * BAR_STRIDE;
    unsigned* top = bar + (size_t)K * BAR_STRIDE;
    double* gp = gpart + (size_t)(epoch & 1u) * (size_t)M * K;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        role = atom_add_acq_rel_u32(sub, 1u) == (unsigned)members * epoch - 1u ? 1 : 0;
    }
    __syncthreads();
    if (role) {
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const double* p = part + (int64_t)m * G + b0;
            double s0 = 0.0, s1 = 0.0;
            int b = 0;
            for (; b + 1 < members; b += 2) {
                s0 += __ldcg(p + b);
                s1 += __ldcg(p + b + 1);
            }
            if (b < members) s0 += __ldcg(p + b);
            if (RBF_IN_RANGE((gp - gpart) + (int64_t)m * K + grp, gpart_len)) gp[(int64_t)m * K + grp] = s0 + s1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            red_add_release_u32(top, 1u);
        }
    }
    if (threadIdx.x == 0) {
        int good = 1;
        long long it = 0;
        const unsigned target = (unsigned)K * epoch;
        while (ld_acquire_u32(top) < target) {
            if (++it > budget) {
                good = 0;
                atomicExch(&stt->info[IN_ERR], (int)RBF_ERR_TIMEOUT);
                atomicExch(&stt->info[IN_DONE], 1);
                break;
            }
        }
        ok = good;
    }
    __syncthreads();
    if (!ok) return false;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const double* p = gp + (int64_t)m * K;
        double s0 = 0.0, s1 = 0.0;
        int q = 0;
        for (; q + 1 < K; q += 2) {
            s0 += __ldcg(p + q);
            s1 += __ldcg(p + q + 1);
        }
        if (q < K) s0 += __ldcg(p + q);
        hs[m] = s0 + s1;
    }
    __syncthreads();
    return true;
}
