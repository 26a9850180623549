// Stopping / lambda network (20 -> 128 -> 128 -> 2, exact-erf GELU, FP32) with
// forward, backward and Adam kernels; the features it reads from the first GKB
// steps; a multi-vector reconstruction used to build its training labels.
//
// Forward: one CTA of 128 threads per tile of 16 samples, thread j owns hidden
// unit j; weights are read coalesced (row-major, unit index fastest) and reused
// across the 16 samples held in shared memory.  Backward: activation gradients
// per tile, then one thread per parameter sums its gradient over the whole
// batch in a fixed order (FP64 accumulation, deterministic).
#include <cfloat>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int NI = RBF_MLP_IN, NH = RBF_MLP_HIDDEN, NO = RBF_MLP_OUT;
constexpr int TS = 16;  // samples per CTA
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NI * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NO, NPAR = OFF_B3 + NO;
static_assert(NPAR == RBF_MLP_PARAMS, "parameter layout");

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// cache (optional): Z1, H1, Z2, H2 [B][NH]
__global__ void __launch_bounds__(NH) k_mlp_fwd(const float* __restrict__ P, const float* __restrict__ X, int B,
                                                float* __restrict__ Y, float* __restrict__ Z1, float* __restrict__ H1,
                                                float* __restrict__ Z2, float* __restrict__ H2) {
    __shared__ float xs[TS][NI];
    __shared__ float h1s[TS][NH];
    __shared__ float h2s[TS][NH];
    __shared__ float red[NH / 32][TS][NO];
    const int s0 = blockIdx.x * TS;
    const int j = threadIdx.x;
    const int ns = min(TS, B - s0);
    for (int q = j; q < TS * NI; q += NH) {
        const int s = q / NI, i = q % NI;
        xs[s][i] = s < ns ? X[(int64_t)(s0 + s) * NI + i] : 0.f;
    }
    __syncthreads();
    float acc[TS];
#pragma unroll
    for (int s = 0; s < TS; ++s) acc[s] = P[OFF_B1 + j];
    for (int i = 0; i < NI; ++i) {
        const float wv = P[OFF_W1 + i * NH + j];
#pragma unroll
        for (int s = 0; s < TS; ++s) acc[s] = fmaf(xs[s][i], wv, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < TS; ++s) {
        const float h = gelu_f(acc[s]);
        h1s[s][j] = h;
        if (Z1 && s < ns) {
            Z1[(int64_t)(s0 + s) * NH + j] = acc[s];
            H1[(int64_t)(s0 + s) * NH + j] = h;
        }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < TS; ++s) acc[s] = P[OFF_B2 + j];
    for (int i = 0; i < NH; ++i) {
        const float wv = P[OFF_W2 + i * NH + j];
#pragma unroll
        for (int s = 0; s < TS; ++s) acc[s] = fmaf(h1s[s][i], wv, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < TS; ++s) {
        const float h = gelu_f(acc[s]);
        h2s[s][j] = h;
        if (Z2 && s < ns) {
            Z2[(int64_t)(s0 + s) * NH + j] = acc[s];
            H2[(int64_t)(s0 + s) * NH + j] = h;
        }
    }
    __syncthreads();
    // output layer: partial products per unit j, reduced across the block
    const float w30 = P[OFF_W3 + j * NO + 0], w31 = P[OFF_W3 + j * NO + 1];
    const int warp = j >> 5, lane = j & 31;
#pragma unroll
    for (int s = 0; s < TS; ++s) {
        float p0 = h2s[s][j] * w30, p1 = h2s[s][j] * w31;
        p0 = warp_sumf(p0);
        p1 = warp_sumf(p1);
        if (lane == 0) {
            red[warp][s][0] = p0;
            red[warp][s][1] = p1;
        }
    }
    __syncthreads();
    if (j < TS * NO) {
        const int s = j / NO, o = j % NO;
        float y = P[OFF_B3 + o];
        for (int w = 0; w < NH / 32; ++w) y += red[w][s][o];
        if (s < ns) Y[(int64_t)(s0 + s) * NO + o] = y;
    }
}

// dY = (Y - T) / B, dZ2, dZ1 per sample; squared-error partial per tile.
__global__ void __launch_bounds__(NH) k_mlp_bwd_act(const float* __restrict__ P, const float* __restrict__ Y,
                                                    const float* __restrict__ T, int B, const float* __restrict__ Z1,
                                                    const float* __restrict__ Z2, float* __restrict__ DY,
                                                    float* __restrict__ DZ1, float* __restrict__ DZ2,
                                                    double* __restrict__ lpart) {
    __shared__ float dys[TS][NO];
    __shared__ float dz2s[TS][NH];
    const int s0 = blockIdx.x * TS;
    const int i = threadIdx.x;
    const int ns = min(TS, B - s0);
    if (i < TS * NO) {
        const int s = i / NO, o = i % NO;
        float d = 0.f;
        if (s < ns) {
            d = (Y[(int64_t)(s0 + s) * NO + o] - T[(int64_t)(s0 + s) * NO + o]);
            DY[(int64_t)(s0 + s) * NO + o] = d / (float)B;
        }
        dys[s][o] = d / (float)B;
    }
    if (i == 0) {
        double l = 0.0;
        for (int s = 0; s < ns; ++s)
            for (int o = 0; o < NO; ++o) {
                const double d = (double)Y[(int64_t)(s0 + s) * NO + o] - (double)T[(int64_t)(s0 + s) * NO + o];
                l += d * d;
            }
        lpart[blockIdx.x] = l;
    }
    __syncthreads();
    const float w30 = P[OFF_W3 + i * NO + 0], w31 = P[OFF_W3 + i * NO + 1];
    for (int s = 0; s < TS; ++s) {
        float dz = 0.f;
        if (s < ns) dz = (dys[s][0] * w30 + dys[s][1] * w31) * gelu_grad_f(Z2[(int64_t)(s0 + s) * NH + i]);
        dz2s[s][i] = dz;
        if (s < ns) DZ2[(int64_t)(s0 + s) * NH + i] = dz;
    }
    __syncthreads();
    // dh1[s][i] = sum_j dz2[s][j] W2[i][j]
    float acc[TS];
#pragma unroll
    for (int s = 0; s < TS; ++s) acc[s] = 0.f;
    for (int jj = 0; jj < NH; ++jj) {
        const float wv = P[OFF_W2 + i * NH + jj];
#pragma unroll
        for (int s = 0; s < TS; ++s) acc[s] = fmaf(dz2s[s][jj], wv, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < TS; ++s)
        if (s < ns) DZ1[(int64_t)(s0 + s) * NH + i] = acc[s] * gelu_grad_f(Z1[(int64_t)(s0 + s) * NH + i]);
}

// One thread per parameter: gradient summed over the batch in sample order.
__global__ void k_mlp_wgrad(const float* __restrict__ X, const float* __restrict__ H1, const float* __restrict__ H2,
                            const float* __restrict__ DY, const float* __restrict__ DZ1, const float* __restrict__ DZ2,
                            int B, float* __restrict__ G) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPAR) return;
    double acc = 0.0;
    if (p < OFF_B1) {
        const int i = p / NH, j = p % NH;
        for (int s = 0; s < B; ++s) acc += (double)X[(int64_t)s * NI + i] * (double)DZ1[(int64_t)s * NH + j];
    } else if (p < OFF_W2) {
        const int j = p - OFF_B1;
        for (int s = 0; s < B; ++s) acc += (double)DZ1[(int64_t)s * NH + j];
    } else if (p < OFF_B2) {
        const int q = p - OFF_W2, i = q / NH, j = q % NH;
        for (int s = 0; s < B; ++s) acc += (double)H1[(int64_t)s * NH + i] * (double)DZ2[(int64_t)s * NH + j];
    } else if (p < OFF_W3) {
        const int j = p - OFF_B2;
        for (int s = 0; s < B; ++s) acc += (double)DZ2[(int64_t)s * NH + j];
    } else if (p < OFF_B3) {
        const int q = p - OFF_W3, i = q / NO, o = q % NO;
        for (int s = 0; s < B; ++s) acc += (double)H2[(int64_t)s * NH + i] * (double)DY[(int64_t)s * NO + o];
    } else {
        const int o = p - OFF_B3;
        for (int s = 0; s < B; ++s) acc += (double)DY[(int64_t)s * NO + o];
    }
    G[p] = (float)acc;
}

__global__ void k_adam(float* __restrict__ P, float* __restrict__ M, float* __restrict__ V,
                       const float* __restrict__ G, float lr, float b1, float b2, float c1, float c2, float eps) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPAR) return;
    const float g = G[p];
    const float m = b1 * M[p] + (1.f - b1) * g;
    const float v = b2 * V[p] + (1.f - b2) * g * g;
    M[p] = m;
    V[p] = v;
    P[p] -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

__global__ void k_sum_parts(const double* __restrict__ parts, int n, double scale, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += parts[q];
        out[0] = s * scale;
    }
}

// Features from the first j GKB steps: [log10 s1, log10(s_i / s1) i=2..10,
// log10(rho_i / beta_1) i=1..10] where rho_i = |C_i y_i - beta_1 e_1| is the
// least-squares residual after i steps (LSQR): rho_i = beta_1 / |u^(i)| with
// u the null vector of C_i^T (u_1 = 1, u_{m+1} = -alpha_m u_m / beta_{m+1}).
// Standardised with (mean, std) when given.
__device__ void stop_features_one(const double* __restrict__ alpha, const double* __restrict__ beta,
                                  const double* __restrict__ sigma, int j, const float* __restrict__ mean,
                                  const float* __restrict__ stdv, float* __restrict__ feat) {
    double f[RBF_MLP_IN];
    const double s1 = sigma[0];
    f[0] = log10(s1);
    for (int i = 1; i < 10; ++i) f[i] = i < j ? log10(fmax(sigma[i], 1e-300) / s1) : -300.0;
    // running log-sum-exp of 2 log|u_m|
    double Lm = 0.0, mx = 0.0, sum = 1.0;  // u_1 = 1
    for (int i = 1; i <= 10; ++i) {
        if (i <= j && beta[i] > 0.0) {
            Lm += log(alpha[i - 1]) - log(beta[i]);
            const double e2 = 2.0 * Lm;
            if (e2 > mx) {
                sum = sum * exp(mx - e2) + 1.0;
                mx = e2;
            } else {
                sum += exp(e2 - mx);
            }
            f[9 + i] = -(0.5 * (mx + log(sum))) / log(10.0);
        } else {
            f[9 + i] = i <= j ? -300.0 : f[9 + i - 1];
        }
    }
    for (int q = 0; q < RBF_MLP_IN; ++q) {
        float v = (float)f[q];
        if (mean && stdv) v = (v - mean[q]) / stdv[q];
        feat[q] = v;
    }
}

__global__ void k_stop_features(const double* __restrict__ alpha, const double* __restrict__ beta,
                                const double* __restrict__ sigma, int j, const float* __restrict__ mean,
                                const float* __restrict__ stdv, float* __restrict__ feat) {
    if (threadIdx.x == 0) stop_features_one(alpha, beta, sigma, j, mean, stdv, feat);
}

// Batched: instance b = blockIdx.x with alpha [B][L], beta [B][L+1], sigma
// [B][L]; instances with fewer than j steps get NaN features.
__global__ void k_stop_features_batch(const double* __restrict__ alpha, const double* __restrict__ beta,
                                      const double* __restrict__ sigma, int L, const int* __restrict__ l_arr, int j,
                                      const float* __restrict__ mean, const float* __restrict__ stdv,
                                      float* __restrict__ feat) {
    const int b = blockIdx.x;
    if (threadIdx.x != 0) return;
    float* out = feat + (size_t)b * RBF_MLP_IN;
    if (l_arr[b] < j) {
        for (int q = 0; q < RBF_MLP_IN; ++q) out[q] = __int_as_float(0x7fc00000);
        return;
    }
    stop_features_one(alpha + (size_t)b * L, beta + (size_t)b * (L + 1), sigma + (size_t)b * L, j, mean, stdv, out);
}

// u[c][t] = sum_j coef[c][j] Phi(|P_t - X_j|) for 8 coefficient vectors per
// grid.z slice (partials over centre chunks in grid.y).
// EM_C coefficient vectors per CTA share each Phi(|P_t - X_j|): 12 FP64-pipe
// operations for Phi plus one FMA per vector.
constexpr int EM_T = 128;
template <int EM_C>
__global__ void __launch_bounds__(EM_T) k_evaluate_many(const double* __restrict__ X, int64_t n,
                                                       const double* __restrict__ coefs, int64_t ldc, int ncoef,
                                                       const double* __restrict__ Pts, int64_t m, double c,
                                                       double scale, int64_t chunk, double* __restrict__ part) {
    __shared__ double sx[EM_T], sy[EM_T], sz[EM_T], sa[EM_C][EM_T];
    const int64_t t = (int64_t)blockIdx.x * EM_T + threadIdx.x;
    const bool active = t < m;
    const double px = active ? Pts[t] : 0.0, py = active ? Pts[m + t] : 0.0, pz = active ? Pts[2 * m + t] : 0.0;
    const int c0 = blockIdx.z * EM_C;
    const int nc = min(EM_C, ncoef - c0);
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = min(n, j0 + chunk);
    const double c2 = c * c;
    double acc[EM_C];
#pragma unroll
    for (int q = 0; q < EM_C; ++q) acc[q] = 0.0;
    for (int64_t jb = j0; jb < j1; jb += EM_T) {
        __syncthreads();
        const int64_t j = jb + threadIdx.x;
        const bool ok = j < j1;
        sx[threadIdx.x] = ok ? X[j] : 0.0;
        sy[threadIdx.x] = ok ? X[n + j] : 0.0;
        sz[threadIdx.x] = ok ? X[2 * n + j] : 0.0;
#pragma unroll
        for (int q = 0; q < EM_C; ++q) sa[q][threadIdx.x] = (ok && q < nc) ? coefs[(int64_t)(c0 + q) * ldc + j] : 0.0;
        __syncthreads();
        const int cnt = (int)min((int64_t)EM_T, j1 - jb);
        for (int r = 0; r < cnt; ++r) {
            const double dx = px - sx[r], dy = py - sy[r], dz = pz - sz[r];
            const double s = fma(dx, dx, fma(dy, dy, fma(dz, dz, c2)));
            const double ph = s * rsqrt_f64(s);
#pragma unroll
            for (int q = 0; q < EM_C; ++q) acc[q] = fma(sa[q][r], ph, acc[q]);
        }
    }
    if (active)
        for (int q = 0; q < nc; ++q) part[((int64_t)blockIdx.y * ncoef + c0 + q) * m + t] = acc[q] * scale;
}

__global__ void k_reduce_many(const double* __restrict__ part, int chunks, int64_t total, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    double s = 0.0;
    for (int q = 0; q < chunks; ++q) s += part[(int64_t)q * total + i];
    out[i] = s;
}

}  // namespace

// ---------------------------------------------------------------------------
static rbf_status mlp_forward_impl(rbf_ctx* ctx, const float* P, const float* X, int B, float* Y, float* cache) {
    float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr;
    if (cache) {
        Z1 = cache;
        H1 = Z1 + (size_t)B * NH;
        Z2 = H1 + (size_t)B * NH;
        H2 = Z2 + (size_t)B * NH;
    }
    k_mlp_fwd<<<(B + TS - 1) / TS, NH, 0, ctx->stream>>>(P, X, B, Y, Z1, H1, Z2, H2);
    RBF_LAUNCHED(ctx, "k_mlp_fwd");
    return RBF_OK;
}

extern "C" rbf_status rbf_mlp_forward(rbf_ctx* ctx, const float* d_params, const float* d_x, int batch, float* d_y) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!d_params || !d_x || !d_y || batch < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_mlp_forward: bad argument");
    return mlp_forward_impl(ctx, d_params, d_x, batch, d_y, nullptr);
}

static rbf_status mlp_grad_impl(rbf_ctx* ctx, const float* P, const float* X, const float* T, int B, float* G,
                                float* h_loss) {
    const int tiles = (B + TS - 1) / TS;
    const size_t need = ws_align((size_t)4 * B * NH * 4) + ws_align((size_t)B * NO * 4) * 2 +
                        ws_align((size_t)2 * B * NH * 4) + ws_align((size_t)(tiles + 1) * 8);
    RBF_TRY(rbf_ws_reserve(ctx, need));
    WsCarve wc(ctx->ws);
    float* cache = wc.take<float>((size_t)4 * B * NH);
    float* Y = wc.take<float>((size_t)B * NO);
    float* DY = wc.take<float>((size_t)B * NO);
    float* DZ = wc.take<float>((size_t)2 * B * NH);
    double* lpart = wc.take<double>((size_t)tiles + 1);
    RBF_TRY(mlp_forward_impl(ctx, P, X, B, Y, cache));
    const float* Z1 = cache;
    const float* H1 = Z1 + (size_t)B * NH;
    const float* Z2 = H1 + (size_t)B * NH;
    const float* H2 = Z2 + (size_t)B * NH;
    float* DZ1 = DZ;
    float* DZ2 = DZ + (size_t)B * NH;
    k_mlp_bwd_act<<<tiles, NH, 0, ctx->stream>>>(P, Y, T, B, Z1, Z2, DY, DZ1, DZ2, lpart);
    RBF_LAUNCHED(ctx, "k_mlp_bwd_act");
    k_mlp_wgrad<<<(NPAR + 255) / 256, 256, 0, ctx->stream>>>(X, H1, H2, DY, DZ1, DZ2, B, G);
    RBF_LAUNCHED(ctx, "k_mlp_wgrad");
    if (h_loss) {
        k_sum_parts<<<1, 32, 0, ctx->stream>>>(lpart, tiles, 1.0 / (2.0 * B), lpart + tiles);
        RBF_LAUNCHED(ctx, "k_sum_parts");
        double l = 0.0;
        RBF_CUDA(ctx, cudaMemcpyAsync(&l, lpart + tiles, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        *h_loss = (float)l;
    }
    return RBF_OK;
}

extern "C" rbf_status rbf_mlp_grad(rbf_ctx* ctx, const float* d_params, const float* d_x, const float* d_t, int batch,
                                   float* d_grad, float* h_loss) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!d_params || !d_x || !d_t || !d_grad || batch < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_mlp_grad: bad argument");
    return mlp_grad_impl(ctx, d_params, d_x, d_t, batch, d_grad, h_loss);
}

extern "C" rbf_status rbf_mlp_adam(rbf_ctx* ctx, float* d_params, float* d_m, float* d_v, const float* d_grad, int t,
                                   float lr) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!d_params || !d_m || !d_v || !d_grad || t < 1) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_mlp_adam: bad argument");
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, t))), c2 = (float)(1.0 / (1.0 - pow(b2, t)));
    k_adam<<<(NPAR + 255) / 256, 256, 0, ctx->stream>>>(d_params, d_m, d_v, d_grad, lr, (float)b1, (float)b2, c1, c2,
                                                        1e-8f);
    RBF_LAUNCHED(ctx, "k_adam");
    return RBF_OK;
}

extern "C" rbf_status rbf_mlp_train_step(rbf_ctx* ctx, float* d_params, float* d_m, float* d_v, int t, float lr,
                                         const float* d_x, const float* d_t, int batch, float* d_grad, float* h_loss) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!d_grad) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_mlp_train_step: gradient buffer required");
    RBF_TRY(mlp_grad_impl(ctx, d_params, d_x, d_t, batch, d_grad, h_loss));
    return rbf_mlp_adam(ctx, d_params, d_m, d_v, d_grad, t, lr);
}

extern "C" rbf_status rbf_stop_features(rbf_ctx* ctx, const rbf_gkb_state* st, int j, const float* d_mean,
                                        const float* d_std, float* d_feat) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!st || !d_feat) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stop_features: NULL argument");
    if (j < 1 || j > 10 || st->steps_done < j)
        return rbf_fail(ctx, RBF_ERR_INVALID, "features need 1 <= j <= 10 completed steps (have %d)", st->steps_done);
    const size_t need = ws_align((size_t)j * 8) + ws_align((size_t)(j + 1) * 8) + ws_align((size_t)j * j * 8) +
                        svd_ws_bytes(j);
    RBF_TRY(rbf_ws_reserve(ctx, need));
    WsCarve wc(ctx->ws);
    double* sigma = wc.take<double>(j);
    double* ftil = wc.take<double>(j + 1);
    double* V = wc.take<double>((size_t)j * j);
    void* svd = (void*)wc.take<char>(svd_ws_bytes(j));
    RBF_TRY(launch_projected_svd(ctx, st->d_alpha, st->d_beta, j, sigma, ftil, V, j, svd));
    k_stop_features<<<1, 32, 0, ctx->stream>>>(st->d_alpha, st->d_beta, sigma, j, d_mean, d_std, d_feat);
    RBF_LAUNCHED(ctx, "k_stop_features");
    return RBF_OK;
}

rbf_status launch_stop_features_batch(rbf_ctx* ctx, const double* alpha, const double* beta, const double* sigma,
                                      int L, const int* d_l, int B, int j, const float* mean, const float* stdv,
                                      float* feat) {
    k_stop_features_batch<<<B, 32, 0, ctx->stream>>>(alpha, beta, sigma, L, d_l, j, mean, stdv, feat);
    RBF_LAUNCHED(ctx, "k_stop_features_batch");
    return RBF_OK;
}

extern "C" rbf_status rbf_evaluate_many(rbf_ctx* ctx, const rbf_operator* op, const double* d_coefs, int64_t ldc,
                                        int ncoef, const double* d_points, int64_t m, double* d_u) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_coefs || !d_points || !d_u || m < 1 || ncoef < 1 || ldc < op->n)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_evaluate_many: bad argument");
    const int64_t n = op->n;
    const int64_t tiles = (m + EM_T - 1) / EM_T;
    // vectors per CTA: the smallest of 1, 2, 4, 8 that holds them all (8 beyond)
    const int em_c = ncoef <= 1 ? 1 : ncoef <= 2 ? 2 : ncoef <= 4 ? 4 : 8;
    const int zs = (ncoef + em_c - 1) / em_c;
    int64_t chunks = ((int64_t)ctx->sm_count * 8 + tiles * zs - 1) / (tiles * zs);
    if (chunks < 1) chunks = 1;
    if ((n + chunks - 1) / chunks < 256) chunks = (n + 255) / 256;
    if (chunks < 1) chunks = 1;
    const int64_t chunk = (n + chunks - 1) / chunks;
    chunks = (n + chunk - 1) / chunk;
    const int64_t total = m * ncoef;
    RBF_TRY(rbf_ws_reserve(ctx, ws_align((size_t)chunks * total * 8)));
    double* part = (double*)ctx->ws;
    const double scale = op->form == RBF_FORM_EPS ? 1.0 / op->c : 1.0;
    const dim3 grid((unsigned)tiles, (unsigned)chunks, (unsigned)zs);
    if (em_c == 1)
        k_evaluate_many<1><<<grid, EM_T, 0, ctx->stream>>>(op->d_nodes, n, d_coefs, ldc, ncoef, d_points, m, op->c,
                                                           scale, chunk, part);
    else if (em_c == 2)
        k_evaluate_many<2><<<grid, EM_T, 0, ctx->stream>>>(op->d_nodes, n, d_coefs, ldc, ncoef, d_points, m, op->c,
                                                           scale, chunk, part);
    else if (em_c == 4)
        k_evaluate_many<4><<<grid, EM_T, 0, ctx->stream>>>(op->d_nodes, n, d_coefs, ldc, ncoef, d_points, m, op->c,
                                                           scale, chunk, part);
    else
        k_evaluate_many<8><<<grid, EM_T, 0, ctx->stream>>>(op->d_nodes, n, d_coefs, ldc, ncoef, d_points, m, op->c,
                                                           scale, chunk, part);
    RBF_LAUNCHED(ctx, "k_evaluate_many");
    k_reduce_many<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(part, (int)chunks, total, d_u);
    RBF_LAUNCHED(ctx, "k_reduce_many");
    return RBF_OK;
}
