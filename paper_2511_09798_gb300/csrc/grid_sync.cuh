// Bounded two-level grid barrier for cooperative kernels (one CTA per slot of
// a cooperative launch).
#pragma once

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
// Grid barrier that also reduces per-CTA partial sums.  part is [M][G] (CTA b
// wrote part[m * G + b]); on a true return h[m] holds, for every m < M,
//   sum over groups q = 0..K-1 (in order) of
//     ( sum over the CTAs b of group q (in order) of part[m * G + b] ),
// and is visible to every CTA.  The last CTA to arrive in a group sums that
// group's columns into gpart[m * K + q]; the last group to arrive sums the K
// group sums into h and then releases the barrier, so the reduction costs no
// barrier of its own.  The order of the additions does not depend on which
// CTA arrives last: the result is deterministic.  Same counters and bounded
// polling as grid_sync.
// ---------------------------------------------------------------------------
static __device__ bool grid_reduce_sync(rbf_dev_state* __restrict__ stt, unsigned* __restrict__ bar, int group,
                                        long long budget, const double* __restrict__ part,
                                        double* __restrict__ gpart, double* __restrict__ h, int M) {
    __shared__ int role;  // bit 0: last of its group, bit 1: last group
    __shared__ int ok;
    const int G = gridDim.x;
    const int K = (G + group - 1) / group;
    const int grp = blockIdx.x / group;
    const int b0 = grp * group;
    const int members = min(group, G - b0);
    unsigned* sub = bar + (size_t)grp * BAR_STRIDE;
    unsigned* top = bar + (size_t)K * BAR_STRIDE;
    volatile unsigned* gen = bar + (size_t)(K + 1) * BAR_STRIDE;
    unsigned g0 = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        g0 = *gen;
        __threadfence();
        role = atomicAdd(sub, 1u) == (unsigned)members - 1 ? 1 : 0;
        __threadfence();
    }
    __syncthreads();
    if (role & 1) {
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            const double* p = part + (int64_t)m * G + b0;
            double s = 0.0;
            for (int b = 0; b < members; ++b) s += __ldcg(p + b);
            gpart[(int64_t)m * K + grp] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(sub, 0u);
            __threadfence();
            role = atomicAdd(top, 1u) == (unsigned)K - 1 ? 3 : 1;
            __threadfence();
        }
        __syncthreads();
        if (role & 2) {
            for (int m = threadIdx.x; m < M; m += blockDim.x) {
                const double* p = gpart + (int64_t)m * K;
                double s = 0.0;
                for (int q = 0; q < K; ++q) s += __ldcg(p + q);
                h[m] = s;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                atomicExch(top, 0u);
                __threadfence();
                atomicAdd((unsigned*)gen, 1u);
            }
        }
    }
    if (threadIdx.x == 0) {
        int good = 1;
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
