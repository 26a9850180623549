// Device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define RBF_FULL_MASK 0xffffffffu

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(RBF_FULL_MASK, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(RBF_FULL_MASK, v, o);
    return v;
}

// 1/sqrt(x) in FP64 for normal x: the hardware's FP64 reciprocal-square-root
// estimate (PTX rsqrt.approx.ftz.f64, no FP32 round trip: two conversions
// fewer on the FP64 pipe than an FP32 estimate) refined by one third-order
// step of the Newton iteration for y = x^{-1/2}: with e = 1 - x y0^2,
// y = y0 (1 + e/2 + 3 e^2 / 8), which cubes the relative error of y0 to below
// FP64 rounding (the collocation entries built on it agree with their FP64
// definition to 2e-15 relative for s from 1e-6 to 3e4 in the tests).
__device__ __forceinline__ double rsqrt_f64(double x) {
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
    double t = x * y0;
    double e = fma(-t, y0, 1.0);
    double c = fma(0.375, e, 0.5);
    return fma(y0 * e, c, y0);
}

__device__ __forceinline__ unsigned sign_bit(double v) {
    return ((unsigned)__double2hiint(v)) >> 31;
}

// Done flag of a GKB run: every GKB kernel returns immediately once set.
__device__ __forceinline__ bool gkb_done(const int* done) {
    return done != nullptr && *(volatile const int*)done != 0;
}

// Flat split of a row-major n x n matrix over W warps (the A z products):
// warp w owns the elements [b_w, b_{w+1}) with b_w = floor(n^2 w / W), its
// column rounded down to a multiple of FLAT_ALIGN (16-byte aligned vector
// loads, full 128-column blocks), so every warp streams the same number of
// entries to within FLAT_ALIGN.  n^2 W stays far below 2^63 for any matrix
// that fits in device memory.
constexpr int64_t FLAT_ALIGN = 128;

__device__ __forceinline__ int64_t flat_bound(int64_t n, int64_t W, int64_t w) {
    if (w >= W) return n * n;
    const int64_t b = n * n * w / W;
    const int64_t r = b / n;
    return r * n + ((b - r * n) & ~(FLAT_ALIGN - 1));
}

// Lambda grid coordinate t_idx = t_lo + idx * step, step = (t_hi - t_lo) /
// (J - 1), rounded as two separate operations (no contraction); the last
// point is exactly t_hi.
__device__ __forceinline__ double grid_t(int idx, int J, double t_lo, double t_hi) {
    if (idx == J - 1) return t_hi;
    const double step = __ddiv_rn(t_hi - t_lo, (double)(J - 1));
    return __dadd_rn(__dmul_rn((double)idx, step), t_lo);
}

// ---- bounds-checked build ---------------------------------------------------
// A library built with -DRBFKR_CHECKED evaluates RBF_IN_RANGE(i, n) as the test
// 0 <= i < n; a failed test records its source line in a device word of the
// translation unit (the first failure is kept) and yields false, so that the
// caller skips the access.  The host collects the words at its synchronisation
// points (rbf_check_take_<unit>, rbf_check_all) and reports RBF_ERR_INTERNAL.
// The checks guard the indexes whose range follows from a planning invariant
// rather than from a test in the kernel (partial-sum slots, shared-memory slab
// sizes, dot-partial and group-sum offsets).  In the normal build the macro is
// `true` and costs nothing.
#ifdef RBFKR_CHECKED
static __device__ unsigned rbf_check_line;
__device__ __forceinline__ bool rbf_in_range(long long i, long long n, unsigned line) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&rbf_check_line, 0u, line);
    return false;
}
#define RBF_IN_RANGE(i, n) rbf_in_range((long long)(i), (long long)(n), __LINE__)
#define RBF_CHECK_READER(unit)                                                              \
    unsigned rbf_check_take_##unit() {                                                      \
        unsigned v = 0, z = 0;                                                              \
        if (cudaMemcpyFromSymbol(&v, rbf_check_line, sizeof(v)) != cudaSuccess) {          \
            cudaGetLastError();                                                             \
            return 0;                                                                       \
        }                                                                                   \
        if (v) cudaMemcpyToSymbol(rbf_check_line, &z, sizeof(z));                           \
        return v;                                                                           \
    }
#else
#define RBF_IN_RANGE(i, n) true
#define RBF_CHECK_READER(unit) \
    unsigned rbf_check_take_##unit() { return 0; }
#endif
