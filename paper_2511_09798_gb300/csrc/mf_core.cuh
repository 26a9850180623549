// Inner loop of the matrix-free FP32 products (single-instance and batched),
// on packed pairs of outputs with the sm_100+ f32x2 instructions.
//
// Entry of row i, column j: s = |X_i - X_j|^2 + c^2, rs = s^{-1/2} and
//   e = rs (a0 rs^2 + a1 + a2 s)
// which is s^{-3/2} (c^2 + 2 s + k^2 s^2) = L Phi for PDE rows ((a0, a1, a2) =
// (c^2, 2, k^2)) and sqrt(s) = Phi for Dirichlet rows ((0, 0, 1)): the two row
// types of A = [H; R] (Sec. 2.1, eqs. H_entries and augmented_system).  When a
// whole tile of entries is Dirichlet the kernel takes e = rs s directly.
//
// Summation nodes sit in shared memory with every value duplicated into both
// halves of a 64-bit pair, so one f32x2 instruction serves two outputs.
#pragma once

#include <cuda_runtime.h>

typedef unsigned long long f2_t;  // two FP32 values: low half = first output of the pair

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float mf_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct MfNode {  // one summation node, each value in both halves
    f2_t xx, yy, zz, ww;
};

__device__ __forceinline__ MfNode mf_node(float x, float y, float z, float w) {
    return MfNode{f2_pack(x, x), f2_pack(y, y), f2_pack(z, z), f2_pack(w, w)};
}

// T[p] += sum over the cnt nodes of the tile of e(o, node) w_node for the NP
// output pairs p.  BND: every entry of the tile is a Dirichlet entry.
template <int NP, bool BND>
__device__ __forceinline__ void mf_tile(const MfNode* __restrict__ tile, int cnt, const f2_t* OX, const f2_t* OY,
                                        const f2_t* OZ, const f2_t* A0, const f2_t* A1, const f2_t* A2, f2_t C2,
                                        f2_t* T) {
#pragma unroll 4
    for (int q = 0; q < cnt; ++q) {
        const MfNode nd = tile[q];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const f2_t dx = f2_sub(OX[p], nd.xx);
            const f2_t dy = f2_sub(OY[p], nd.yy);
            const f2_t dz = f2_sub(OZ[p], nd.zz);
            f2_t s = f2_fma(dz, dz, C2);
            s = f2_fma(dy, dy, s);
            s = f2_fma(dx, dx, s);
            float s0, s1;
            f2_unpack(s, s0, s1);
            const f2_t rs = f2_pack(mf_rsqrt(s0), mf_rsqrt(s1));
            f2_t e;
            if (BND) {
                e = f2_mul(rs, s);
            } else {
                f2_t g = f2_fma(A2[p], s, A1[p]);
                g = f2_fma(A0[p], f2_mul(rs, rs), g);
                e = f2_mul(rs, g);
            }
            T[p] = f2_fma(e, nd.ww, T[p]);
        }
    }
}
