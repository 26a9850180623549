// Matrix-free FP32 products (single-instance and batched) by tile pairs, on
// packed pairs of rows with the sm_100+ f32x2 instructions.
//
// Entry of row i, column j: s = |X_i - X_j|^2 + c^2, rs = s^{-1/2} and
//   e = rs (a0 rs^2 + a1 + a2 s)
// which is s^{-3/2} (c^2 + 2 s + k^2 s^2) = L Phi for PDE rows ((a0, a1, a2) =
// (c^2, 2, k^2)) and sqrt(s) = Phi for Dirichlet rows ((0, 0, 1)): the two row
// types of A = [H; R] (Sec. 2.1, eqs. H_entries and augmented_system); a
// Dirichlet entry is taken as rs s.  s and rs are symmetric in (i, j), so one
// evaluation per node pair serves A_ij and A_ji.
//
// Column nodes sit in shared memory with every value duplicated into both
// halves of a 64-bit pair, so one f32x2 instruction serves two rows.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

// ---------------------------------------------------------------------------
// Tile-pair products (single-instance k_mf_sym and the batched kernel).
// ---------------------------------------------------------------------------
constexpr int MS_W = 4;                          // warps per CTA, splitting the tile's columns
enum { MS_INT = 0, MS_BND = 1, MS_MIX = 2 };     // row / column type of a range of nodes

__device__ __forceinline__ int ms_type(int64_t lo, int64_t hi, int64_t ni) {
    return hi <= ni ? MS_INT : (lo >= ni ? MS_BND : MS_MIX);
}

// 32 staged columns against the lane's NP row pairs.  Entries of the row's
// type: eR; of the column's type: eC.  The own side (outputs = the lane's rows)
// takes T=0: A_ij = eR, T=1: A_ji = eC, times x_j; with SYM the other side
// (outputs = the columns) takes the other one times x_i, summed over the
// lane's rows into colpart[q][lane].
template <int TRANS, bool SYM, int RT, int CT, int NP>
__device__ __forceinline__ void ms_cols(const MfNode* __restrict__ cols, float (*colpart)[33], int lane,
                                        const f2_t* OX, const f2_t* OY, const f2_t* OZ, const f2_t* XI,
                                        unsigned imask, f2_t C2, f2_t K2, f2_t TWO, int64_t cb, int64_t ni,
                                        f2_t* T) {
    constexpr bool useR = SYM || TRANS == 0;
    constexpr bool useC = SYM || TRANS == 1;
    constexpr bool needL = (useR && RT != MS_BND) || (useC && CT != MS_BND);
    constexpr bool needP = (useR && RT != MS_INT) || (useC && CT != MS_INT);
#pragma unroll 2
    for (int q = 0; q < 32; ++q) {
        const MfNode nd = cols[q];
        const bool cint = CT == MS_INT || (CT == MS_MIX && cb + q < ni);
        f2_t CA = 0ull;
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
            f2_t eL = 0ull, eP = 0ull, eR;
            if constexpr (needL) eL = f2_mul(rs, f2_fma(C2, f2_mul(rs, rs), f2_fma(K2, s, TWO)));
            if constexpr (needP) eP = f2_mul(rs, s);
            if constexpr (RT == MS_MIX) {  // bit 2p + h of imask: row 2p + h is a PDE row
                float l0, l1, p0, p1;
                f2_unpack(eL, l0, l1);
                f2_unpack(eP, p0, p1);
                eR = f2_pack((imask >> (2 * p)) & 1u ? l0 : p0, (imask >> (2 * p + 1)) & 1u ? l1 : p1);
            } else {
                eR = RT == MS_INT ? eL : eP;
            }
            const f2_t eC = cint ? eL : eP;
            T[p] = f2_fma(TRANS == 0 ? eR : eC, nd.ww, T[p]);
            if constexpr (SYM) CA = p == 0 ? f2_mul(TRANS == 0 ? eC : eR, XI[p]) : f2_fma(TRANS == 0 ? eC : eR, XI[p], CA);
        }
        if constexpr (SYM) {
            float lo, hi;
            f2_unpack(CA, lo, hi);
            colpart[q][lane] = lo + hi;
        }
    }
}

template <int TRANS, bool SYM, int NP>
__device__ __forceinline__ void ms_dispatch(int rt, int ct, const MfNode* cols, float (*colpart)[33], int lane,
                                            const f2_t* OX, const f2_t* OY, const f2_t* OZ, const f2_t* XI,
                                            unsigned imask, f2_t C2, f2_t K2, f2_t TWO, int64_t cb, int64_t ni,
                                            f2_t* T) {
    // without SYM only one of the two types matters
    if (!SYM && TRANS == 0) ct = MS_INT;
    if (!SYM && TRANS == 1) rt = MS_INT;
#define MS_CASE(R_, C_)                                                                                        \
    case R_ * 3 + C_:                                                                                          \
        ms_cols<TRANS, SYM, R_, C_, NP>(cols, colpart, lane, OX, OY, OZ, XI, imask, C2, K2, TWO, cb, ni, T);    \
        break;
    switch (rt * 3 + ct) {
        MS_CASE(MS_INT, MS_INT)
        MS_CASE(MS_INT, MS_BND)
        MS_CASE(MS_INT, MS_MIX)
        MS_CASE(MS_BND, MS_INT)
        MS_CASE(MS_BND, MS_BND)
        MS_CASE(MS_BND, MS_MIX)
        MS_CASE(MS_MIX, MS_INT)
        MS_CASE(MS_MIX, MS_BND)
        MS_CASE(MS_MIX, MS_MIX)
        default: break;
    }
#undef MS_CASE
}

// Tile (I, J) of blocks of B = 32 R nodes, by one CTA of MS_W warps: rows
// I*B + lane + 32 r (r < R).  Writes the contributions to the outputs of block
// I into slot J (part[J][.]) and, for I < J, those to the outputs of block J
// into slot I.  X: FP32 node coordinates SoA [3][n]; x32: the FP32 input.
// SlotT double: a slot holds the FP64 value of the FP32 run times scale;
// SlotT float: the FP32 run itself, unscaled (the batched half-step adds the
// slots with compensated FP32 sums and applies scale).
template <int TRANS, int R, typename SlotT = double>
__device__ __forceinline__ void ms_tile_product(const float* __restrict__ X, int64_t n, int64_t ni, float c2,
                                                float k2, double scale, const float* __restrict__ x32, int64_t I,
                                                int64_t J, SlotT* __restrict__ part) {
    constexpr int NP = R / 2, B = 32 * R, CW = B / MS_W;  // CW columns per warp
    static_assert(CW % 32 == 0, "a warp takes whole groups of 32 columns");
    __shared__ MfNode cols[MS_W][32];
    __shared__ float colpart[MS_W][32][33];
    __shared__ float own[MS_W][R][32];
    const bool sym = I != J;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = I * B, col0 = J * B;
    const int rt = ms_type(row0, row0 + B, ni);
    f2_t OX[NP], OY[NP], OZ[NP], XI[NP], T[NP];
    unsigned imask = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float cx[2], cy[2], cz[2], xv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = row0 + lane + 32 * (2 * p + h);
            const bool ok = i < n;
            cx[h] = ok ? X[i] : 0.f;
            cy[h] = ok ? X[n + i] : 0.f;
            cz[h] = ok ? X[2 * n + i] : 0.f;
            xv[h] = ok ? x32[i] : 0.f;
            if (i < ni) imask |= 1u << (2 * p + h);
        }
        OX[p] = f2_pack(cx[0], cx[1]);
        OY[p] = f2_pack(cy[0], cy[1]);
        OZ[p] = f2_pack(cz[0], cz[1]);
        XI[p] = f2_pack(xv[0], xv[1]);
        T[p] = 0ull;
    }
    const f2_t C2 = f2_pack(c2, c2), K2 = f2_pack(k2, k2), TWO = f2_pack(2.f, 2.f);
    const bool scaled = scale != 1.0;
    for (int g = 0; g < CW / 32; ++g) {
        const int64_t cb = col0 + warp * CW + g * 32;
        {
            const int64_t j = cb + lane;
            const bool ok = j < n;
            cols[warp][lane] = ok ? mf_node(X[j], X[n + j], X[2 * n + j], x32[j]) : mf_node(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        const int ct = ms_type(cb, cb + 32, ni);
        if (sym)
            ms_dispatch<TRANS, true, NP>(rt, ct, cols[warp], colpart[warp], lane, OX, OY, OZ, XI, imask, C2, K2, TWO,
                                         cb, ni, T);
        else
            ms_dispatch<TRANS, false, NP>(rt, ct, cols[warp], colpart[warp], lane, OX, OY, OZ, XI, imask, C2, K2,
                                          TWO, cb, ni, T);
        __syncwarp();
        if (sym) {
            // column cb + lane: the sum over the warp's 32 R rows (lanes m, m + 4,
            // ... in four running sums, then combined in a fixed order)
            float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int m = 0; m < 32; ++m) v[m & 3] += colpart[warp][lane][m];
            const float vs = (v[0] + v[1]) + (v[2] + v[3]);
            const int64_t j = cb + lane;
            if (j < n) {
                if constexpr (sizeof(SlotT) == sizeof(float)) part[I * n + j] = vs;
                else part[I * n + j] = scaled ? (double)vs * scale : (double)vs;
            }
            __syncwarp();
        }
    }
    // row sums: the warps' FP32 partials added in order (FP32: B products in all)
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float t0, t1;
        f2_unpack(T[p], t0, t1);
        own[warp][2 * p][lane] = t0;
        own[warp][2 * p + 1][lane] = t1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < B; e += MS_W * 32) {
        const int r = e >> 5, l = e & 31;
        const int64_t i = row0 + l + 32 * r;
        float acc = 0.f;
#pragma unroll
        for (int w = 0; w < MS_W; ++w) acc += own[w][r][l];
        if (i < n) {
            if constexpr (sizeof(SlotT) == sizeof(float)) part[J * n + i] = acc;
            else part[J * n + i] = scaled ? (double)acc * scale : (double)acc;
        }
    }
}

