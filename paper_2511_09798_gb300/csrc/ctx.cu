// Context, workspace, errors, timings and operator validation.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "common.cuh"
#include "internal.h"

rbf_status rbf_fail(rbf_ctx* ctx, rbf_status st, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

rbf_status rbf_ws_reserve(rbf_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return RBF_OK;
    if (ctx->opt.workspace_cap > 0 && bytes > (size_t)ctx->opt.workspace_cap)
        return rbf_fail(ctx, RBF_ERR_OOM, "workspace of %zu bytes exceeds the cap of %lld bytes",
                        bytes, (long long)ctx->opt.workspace_cap);
    if (ctx->ws) {
        RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        RBF_CUDA(ctx, cudaFree(ctx->ws));
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    size_t grow = bytes + bytes / 4;
    cudaError_t e = cudaMalloc(&ctx->ws, grow);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return rbf_fail(ctx, RBF_ERR_OOM, "cudaMalloc of %zu workspace bytes failed: %s", grow,
                        cudaGetErrorString(e));
    }
    ctx->ws_bytes = grow;
    return RBF_OK;
}

// Product-launch timing: a lane records on its own stream into its owner's
// event slots (the owner's base event precedes every lane's work, see
// rbf_lanes_fork), so that busy intervals of all lanes share one time origin.
int rbf_prod_begin(rbf_ctx* ctx, int kind, cudaStream_t s) {
    rbf_ctx* o = ctx->owner ? ctx->owner : ctx;
    if (!s) s = ctx->stream;
    o->ptotal[kind]++;
    if (!(o->opt.timing & 2) || !o->pev || o->pcount[kind] >= rbf_ctx::PMAX) return -1;
    if (!o->pbase_set) {
        cudaEventRecord(o->pbase, s);
        o->pbase_set = true;
    }
    const int slot = o->pcount[kind]++;
    cudaEventRecord(o->pev[((size_t)kind * rbf_ctx::PMAX + slot) * 2], s);
    return slot;
}

void rbf_prod_end(rbf_ctx* ctx, int kind, int slot, cudaStream_t s) {
    if (slot < 0) return;
    rbf_ctx* o = ctx->owner ? ctx->owner : ctx;
    cudaEventRecord(o->pev[((size_t)kind * rbf_ctx::PMAX + slot) * 2 + 1], s ? s : ctx->stream);
}

rbf_status rbf_lane(rbf_ctx* ctx, int i, rbf_ctx** out) {
    if (!ctx->lane[i]) {
        rbf_options o = ctx->opt;
        o.timing = 0;  // a lane's product timings go to its owner; no per-phase timers
        cudaStream_t s = nullptr;
        int prev = 0;  // the caller's current device is restored below
        RBF_CUDA(ctx, cudaGetDevice(&prev));
        RBF_CUDA(ctx, cudaSetDevice(ctx->device));
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        rbf_ctx* l = nullptr;
        const bool made = e == cudaSuccess && rbf_create(&l, ctx->device, s, &o) == RBF_OK;
        cudaSetDevice(prev);
        if (!made) {
            if (s) cudaStreamDestroy(s);
            return rbf_fail(ctx, RBF_ERR_CUDA, "creating lane %d failed", i);
        }
        l->own_stream = true;
        l->owner = ctx;
        ctx->lane[i] = l;
    }
    *out = ctx->lane[i];
    return RBF_OK;
}

rbf_status rbf_many_slots(rbf_ctx* ctx, int count) {
    if (count <= ctx->h_many_cap) return RBF_OK;
    if (ctx->h_many) {
        RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFreeHost(ctx->h_many);
        ctx->h_many = nullptr;
        ctx->h_many_cap = 0;
    }
    RBF_CUDA(ctx, cudaMallocHost(&ctx->h_many, sizeof(rbf_dev_state) * (size_t)count));
    ctx->h_many_cap = count;
    return RBF_OK;
}

rbf_status rbf_lanes_fork(rbf_ctx* ctx, int lanes) {
    if (ctx->pev && !ctx->pbase_set) {  // product timing: the origin precedes all lanes
        RBF_CUDA(ctx, cudaEventRecord(ctx->pbase, ctx->stream));
        ctx->pbase_set = true;
    }
    RBF_CUDA(ctx, cudaEventRecord(ctx->sync_ev, ctx->stream));
    for (int i = 0; i < lanes; ++i) {
        rbf_ctx* l = nullptr;
        RBF_TRY(rbf_lane(ctx, i, &l));
        RBF_CUDA(ctx, cudaStreamWaitEvent(l->stream, ctx->sync_ev, 0));
    }
    return RBF_OK;
}

rbf_status rbf_lanes_join(rbf_ctx* ctx, int lanes) {
    rbf_status st = RBF_OK;
    for (int i = 0; i < lanes; ++i) {
        rbf_ctx* l = ctx->lane[i];
        if (!l) continue;
        ctx->launches += l->launches;
        l->launches = 0;
        cudaError_t e = cudaEventRecord(l->sync_ev, l->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, l->sync_ev, 0);
        if (e != cudaSuccess && st == RBF_OK)
            st = rbf_fail(ctx, RBF_ERR_CUDA, "joining lane %d failed: %s", i, cudaGetErrorString(e));
    }
    return st;
}

void rbf_timer_start(rbf_ctx* ctx) {
    if (ctx->opt.timing & 1) cudaEventRecord(ctx->ev[0], ctx->stream);
}

double rbf_timer_stop(rbf_ctx* ctx) {
    if (!(ctx->opt.timing & 1)) return 0.0;
    cudaEventRecord(ctx->ev[1], ctx->stream);
    cudaEventSynchronize(ctx->ev[1]);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    return (double)ms;
}

RBF_CHECK_READER(ctx)

rbf_status rbf_sync_all(rbf_ctx* ctx) {
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < rbf_ctx::MAX_LANES; ++i)
        if (ctx->lane[i]) RBF_CUDA(ctx, cudaStreamSynchronize(ctx->lane[i]->stream));
    cudaStream_t bs = rbf_batch_stream(ctx);
    if (bs) RBF_CUDA(ctx, cudaStreamSynchronize(bs));
    return RBF_OK;
}

rbf_status rbf_check_all(rbf_ctx* ctx) {
    struct Unit {
        const char* name;
        unsigned (*take)();
    };
    const Unit units[] = {{"ctx.cu", rbf_check_take_ctx},         {"gemv.cu", rbf_check_take_gemv},
                          {"gkb.cu", rbf_check_take_gkb},         {"batch.cu", rbf_check_take_batch},
                          {"select.cu", rbf_check_take_select},   {"assemble.cu", rbf_check_take_assemble},
                          {"mf.cu", rbf_check_take_mf},           {"fx.cu", rbf_check_take_fx}};
    rbf_status st = RBF_OK;
    for (const Unit& u : units) {
        const unsigned line = u.take();
        if (line && st == RBF_OK)
            st = rbf_fail(ctx, RBF_ERR_INTERNAL, "device index check failed in %s at line %u", u.name, line);
    }
    return st;
}

namespace {
// Exercises the checked-build plumbing: one index test that fails by
// construction (5 outside [0, 3)); no memory is accessed either way.
__global__ void k_check_selftest(int* out) {
    if (!RBF_IN_RANGE(5, 3)) out[0] = 1;
}
}  // namespace

extern "C" {

int rbf_checked_build(void) {
#ifdef RBFKR_CHECKED
    return 1;
#else
    return 0;
#endif
}

rbf_status rbf_check(rbf_ctx* ctx) {
    RbfRange range_("rbf_check");
    if (!ctx) return RBF_ERR_INVALID;
    RBF_TRY(rbf_sync_all(ctx));
    return rbf_check_all(ctx);
}

rbf_status rbf_check_selftest(rbf_ctx* ctx) {
    if (!ctx) return RBF_ERR_INVALID;
    k_check_selftest<<<1, 1, 0, ctx->stream>>>(&ctx->d_state->info[IN_SCRATCH]);
    RBF_LAUNCHED(ctx, "k_check_selftest");
    return RBF_OK;
}

rbf_status rbf_create(rbf_ctx** out, int device, void* cuda_stream, const rbf_options* opt) {
    if (!out) return RBF_ERR_INVALID;
    *out = nullptr;
    rbf_ctx* ctx = new rbf_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (opt) ctx->opt = *opt;
    if (ctx->opt.grid_j <= 0) ctx->opt.grid_j = 321;
    if (ctx->opt.grid_j < 3) {  // the L-curve needs interior grid points, the grid step J - 1 > 0
        delete ctx;
        return RBF_ERR_INVALID;
    }
    if (!(ctx->opt.grid_t_lo < ctx->opt.grid_t_hi)) {
        ctx->opt.grid_t_lo = -16.0;
        ctx->opt.grid_t_hi = 0.0;
    }
    if (ctx->opt.breakdown_factor <= 0) ctx->opt.breakdown_factor = 64.0;
    if (ctx->opt.cluster_tol <= 0) ctx->opt.cluster_tol = 1e-3;
    if (ctx->opt.wait_budget <= 0) ctx->opt.wait_budget = 1LL << 23;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_state, sizeof(rbf_dev_state));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_state, sizeof(rbf_dev_state));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_state, 0, sizeof(rbf_dev_state));
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev[1]);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->pbase);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->sync_ev, cudaEventDisableTiming);
    if (e == cudaSuccess && (ctx->opt.timing & 2)) {
        const size_t ne = (size_t)rbf_ctx::PKINDS * rbf_ctx::PMAX * 2;
        ctx->pev = new cudaEvent_t[ne]();
        for (size_t i = 0; i < ne && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->pev[i]);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        rbf_destroy(ctx);
        return RBF_ERR_CUDA;
    }
    *out = ctx;
    return RBF_OK;
}

rbf_status rbf_get_counters(rbf_ctx* ctx, rbf_counters* out, int reset) {
    if (!ctx || !out) return RBF_ERR_INVALID;
    out->launches = ctx->launches;
    for (int t = 0; t < 2; ++t) {
        out->product_launches[t] = ctx->pcount[t];
        out->product_ms[t] = 0.0;
    }
    out->product_busy_ms = 0.0;
    out->reorth_launches = ctx->pcount[2];
    out->reorth_ms = 0.0;
    if (ctx->pev && ctx->pcount[2]) {
        RBF_TRY(rbf_sync_all(ctx));
        for (int i = 0; i < ctx->pcount[2]; ++i) {
            float ms = 0.f;
            const size_t b = ((size_t)2 * rbf_ctx::PMAX + i) * 2;
            RBF_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->pev[b], ctx->pev[b + 1]));
            out->reorth_ms += ms;
        }
    }
    if (ctx->pev && (ctx->pcount[0] || ctx->pcount[1])) {
        RBF_TRY(rbf_sync_all(ctx));
        std::vector<std::pair<double, double>> iv;
        iv.reserve((size_t)ctx->pcount[0] + ctx->pcount[1]);
        for (int t = 0; t < 2; ++t)
            for (int i = 0; i < ctx->pcount[t]; ++i) {
                float ms = 0.f, t0 = 0.f, t1 = 0.f;
                const size_t b = ((size_t)t * rbf_ctx::PMAX + i) * 2;
                RBF_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->pev[b], ctx->pev[b + 1]));
                RBF_CUDA(ctx, cudaEventElapsedTime(&t0, ctx->pbase, ctx->pev[b]));
                RBF_CUDA(ctx, cudaEventElapsedTime(&t1, ctx->pbase, ctx->pev[b + 1]));
                out->product_ms[t] += ms;
                iv.emplace_back((double)t0, (double)t1);
            }
        // union of the launch intervals: time during which any product ran
        std::sort(iv.begin(), iv.end());
        double cs = iv[0].first, ce = iv[0].second;
        for (size_t i = 1; i < iv.size(); ++i) {
            if (iv[i].first > ce) {
                out->product_busy_ms += ce - cs;
                cs = iv[i].first;
                ce = iv[i].second;
            } else if (iv[i].second > ce) {
                ce = iv[i].second;
            }
        }
        out->product_busy_ms += ce - cs;
    }
    if (reset) {
        ctx->launches = 0;
        for (int t = 0; t < rbf_ctx::PKINDS; ++t) ctx->pcount[t] = 0, ctx->ptotal[t] = 0;
        ctx->pbase_set = false;
    }
    return RBF_OK;
}

rbf_status rbf_destroy(rbf_ctx* ctx) {
    if (!ctx) return RBF_OK;
    for (auto& l : ctx->lane) {
        rbf_destroy(l);
        l = nullptr;
    }
    if (ctx->stream || ctx->d_state) cudaStreamSynchronize(ctx->stream);
    rbf_batch_state_free(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_state) cudaFree(ctx->d_state);
    if (ctx->h_state) cudaFreeHost(ctx->h_state);
    for (auto& ev : ctx->ev)
        if (ev) cudaEventDestroy(ev);
    if (ctx->pbase) cudaEventDestroy(ctx->pbase);
    if (ctx->sync_ev) cudaEventDestroy(ctx->sync_ev);
    if (ctx->h_many) cudaFreeHost(ctx->h_many);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->pev) {
        for (size_t i = 0; i < (size_t)rbf_ctx::PKINDS * rbf_ctx::PMAX * 2; ++i)
            if (ctx->pev[i]) cudaEventDestroy(ctx->pev[i]);
        delete[] ctx->pev;
    }
    delete ctx;
    return RBF_OK;
}

const char* rbf_last_error(const rbf_ctx* ctx) { return ctx ? ctx->err : "null context"; }

rbf_status rbf_get_timings(const rbf_ctx* ctx, rbf_timings* out) {
    if (!ctx || !out) return RBF_ERR_INVALID;
    *out = ctx->tim;
    return RBF_OK;
}

size_t rbf_workspace_bytes(const rbf_ctx* ctx, int64_t n, int steps, int storage, int precision) {
    if (!ctx || n <= 0 || steps <= 0) return 0;
    size_t a = gkb_ws_bytes(ctx, n, steps, precision);
    rbf_operator fake{};  // the fixed-point copies of an FP64 assembled operator (lda padded to even)
    fake.n = n;
    fake.lda = (n + 1) & ~(int64_t)1;
    fake.storage = storage;
    fake.precision = precision;
    if (fx_eligible(ctx, &fake)) a += fx_ws_bytes(&fake);
    size_t b = svd_ws_bytes(steps) + select_ws_bytes(ctx, steps);
    size_t c = gemv_ws_bytes(ctx, n) + ws_align((size_t)n * 8) * 2 + 4096;
    size_t m = a > b ? a : b;
    return m > c ? m : c;
}

rbf_status rbf_operator_init(rbf_ctx* ctx, rbf_operator* op, const double* d_nodes, int64_t n,
                             int64_t n_interior, double c, double k, int storage, int precision,
                             int form, void* d_A, int64_t lda) {
    if (!ctx) return RBF_ERR_INVALID;
    if (!op) return rbf_fail(ctx, RBF_ERR_INVALID, "op is NULL");
    if (!d_nodes) return rbf_fail(ctx, RBF_ERR_INVALID, "d_nodes is NULL");
    if (n <= 0) return rbf_fail(ctx, RBF_ERR_INVALID, "n must be positive (got %lld)", (long long)n);
    if (n > ((int64_t)1 << 31) - 1)
        return rbf_fail(ctx, RBF_ERR_INVALID, "n too large (%lld)", (long long)n);
    if (n_interior < 0 || n_interior > n)
        return rbf_fail(ctx, RBF_ERR_INVALID, "n_interior %lld outside [0, n]", (long long)n_interior);
    if (!(c > 0.0)) return rbf_fail(ctx, RBF_ERR_INVALID, "c must be positive");
    if (!(k >= 0.0)) return rbf_fail(ctx, RBF_ERR_INVALID, "k must be non-negative");
    if (storage != RBF_ASSEMBLED && storage != RBF_MATRIX_FREE)
        return rbf_fail(ctx, RBF_ERR_INVALID, "unknown storage %d", storage);
    if (precision != RBF_FP64 && precision != RBF_MIXED)
        return rbf_fail(ctx, RBF_ERR_INVALID, "unknown precision %d", precision);
    if (form != RBF_FORM_C && form != RBF_FORM_EPS)
        return rbf_fail(ctx, RBF_ERR_INVALID, "unknown form %d", form);
    if (storage == RBF_ASSEMBLED) {
        if (!d_A) return rbf_fail(ctx, RBF_ERR_INVALID, "assembled operator needs d_A");
        if (lda < n) return rbf_fail(ctx, RBF_ERR_INVALID, "lda %lld < n %lld", (long long)lda, (long long)n);
        int vec = precision == RBF_FP64 ? 2 : 4;
        if (lda % vec != 0 || ((uintptr_t)d_A & 15u) != 0)
            return rbf_fail(ctx, RBF_ERR_INVALID,
                            "d_A must be 16-byte aligned and lda a multiple of %d elements", vec);
    }
    op->d_nodes = d_nodes;
    op->n = n;
    op->n_interior = n_interior;
    op->c = c;
    op->k = k;
    op->storage = storage;
    op->precision = precision;
    op->form = form;
    op->d_A = storage == RBF_ASSEMBLED ? d_A : nullptr;
    op->lda = storage == RBF_ASSEMBLED ? lda : 0;
    return RBF_OK;
}

rbf_status rbf_assemble(rbf_ctx* ctx, const rbf_operator* op) {
    RbfRange range_("rbf_assemble");
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || op->storage != RBF_ASSEMBLED || !op->d_A)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_assemble needs an assembled operator");
    rbf_timer_start(ctx);
    RBF_TRY(launch_assemble(ctx, op));
    ctx->tim.assemble_ms = rbf_timer_stop(ctx);
    return RBF_OK;
}

rbf_status rbf_evaluate(rbf_ctx* ctx, const rbf_operator* op, const double* d_coef,
                        const double* d_points, int64_t m, double* d_u) {
    RbfRange range_("rbf_evaluate");
    if (!ctx) return RBF_ERR_INVALID;
    if (!op || !d_coef || !d_points || !d_u)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_evaluate: NULL argument");
    if (m <= 0) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_evaluate: m must be positive");
    rbf_timer_start(ctx);
    RBF_TRY(launch_evaluate(ctx, op, d_coef, d_points, m, d_u));
    ctx->tim.evaluate_ms = rbf_timer_stop(ctx);
    return RBF_OK;
}

}  // extern "C"
