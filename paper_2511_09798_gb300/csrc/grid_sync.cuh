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

