// Throughput probes of the FP64 units, used for the roofline peak of the FP64
// products (not part of the solver path).  Each probe keeps every SM busy with
// independent work and is timed with CUDA events on the context stream:
//   mode 0  FP64 FMA: 8 independent fma chains per thread
//   mode 1  FP64 MMA: mma.sync m8n8k4 (f64 in, f64 accumulate), 4 independent
//           accumulators per warp
//   mode 2  both in every warp: one MMA and 8 FMA per iteration
// The result is the operation count divided by the event time; per SM per
// clock it needs the SM clock, which the caller samples while the probe runs.
#include "internal.h"

namespace {

constexpr int PR_THREADS = 256;

__device__ __forceinline__ void dmma_m8n8k4(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

template <int MODE>
__global__ void __launch_bounds__(PR_THREADS) k_probe_fp64(long long iters, double seed, double* __restrict__ out) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = seed + 0.001 * (threadIdx.x + u);
    double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    const double a = 1.0 - 1e-12 * seed, b = 1e-9 * seed;
    for (long long it = 0; it < iters; ++it) {
        if (MODE != 0) {
#pragma unroll
            for (int q = 0; q < (MODE == 1 ? 4 : 1); ++q) dmma_m8n8k4(acc[q], a + q, b + q);
        }
        if (MODE != 1) {
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
#pragma unroll
    for (int q = 0; q < 4; ++q) s += acc[q][0] + acc[q][1];
    // a store the compiler cannot drop, taken by no thread for a positive seed
    if (s == -1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" rbf_status rbf_probe_fp64(rbf_ctx* ctx, int mode, long long iters, double* d_out, double* ms,
                                     double* flops) {
    RbfRange range_("rbf_probe_fp64");
    if (!ctx) return RBF_ERR_INVALID;
    if (mode < 0 || mode > 2 || iters < 1 || !d_out || !ms || !flops)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_probe_fp64: mode 0..2, iters >= 1, outputs required");
    int per_sm = 0;
    const void* fn = mode == 0 ? (const void*)k_probe_fp64<0> : mode == 1 ? (const void*)k_probe_fp64<1>
                                                                          : (const void*)k_probe_fp64<2>;
    RBF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PR_THREADS, 0));
    const int grid = ctx->sm_count * (per_sm < 1 ? 1 : per_sm);
    cudaStream_t s = ctx->stream;
    RBF_CUDA(ctx, cudaEventRecord(ctx->ev[0], s));
    if (mode == 0) k_probe_fp64<0><<<grid, PR_THREADS, 0, s>>>(iters, 1.0, d_out);
    else if (mode == 1) k_probe_fp64<1><<<grid, PR_THREADS, 0, s>>>(iters, 1.0, d_out);
    else k_probe_fp64<2><<<grid, PR_THREADS, 0, s>>>(iters, 1.0, d_out);
    RBF_LAUNCHED(ctx, "k_probe_fp64");
    RBF_CUDA(ctx, cudaEventRecord(ctx->ev[1], s));
    RBF_CUDA(ctx, cudaEventSynchronize(ctx->ev[1]));
    float t = 0.f;
    RBF_CUDA(ctx, cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]));
    *ms = (double)t;
    const double threads = (double)grid * PR_THREADS, warps = threads / 32.0;
    const double fma_flops = mode == 1 ? 0.0 : threads * (double)iters * 8.0 * 2.0;
    const double mma_flops = mode == 0 ? 0.0 : warps * (double)iters * (mode == 1 ? 4.0 : 1.0) * 2.0 * 8 * 8 * 4;
    *flops = fma_flops + mma_flops;
    return RBF_OK;
}
