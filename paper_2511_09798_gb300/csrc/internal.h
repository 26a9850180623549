// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>

#include "rbfkr.h"

// Device-side small state, one block per context (lives in the context's
// fixed allocation, never in the growable workspace).
struct rbf_dev_state {
    int info[8];      // 0 steps_done, 1 breakdown, 2 done flag, 3 error code, 4 cur step
    double scal[16];  // see SC_* below
    float mlp[64];    // learned stop: features [0, 20), network output [32, 34)
};
enum {
    SC_CHAT0 = 0,   // c_hat double buffer slot 0
    SC_CHAT1 = 1,   // slot 1
    SC_INV_BETA = 2,
    SC_BETA = 3,
    SC_INV_ALPHA = 4,
    SC_ALPHA = 5,
    SC_LAMBDA = 6,  // chosen lambda
    SC_SIGMA1 = 7,
    SC_FTIL_LAST = 8,
    SC_ETA = 9,     // |y| of the last projected solve
    SC_RHO = 10,    // projected residual of the last projected solve
};
enum { IN_STEPS = 0, IN_BREAK = 1, IN_DONE = 2, IN_ERR = 3, IN_INDEX = 4, IN_RANK = 5, IN_SCRATCH = 7 };

// Named NVTX range around a library call, shown on Nsight timelines; a
// no-op unless a profiling tool is attached.  Scoped, so that a call that
// returns early with an error still closes its range.
struct RbfRange {
    explicit RbfRange(const char* name) { nvtxRangePushA(name); }
    ~RbfRange() { nvtxRangePop(); }
    RbfRange(const RbfRange&) = delete;
    RbfRange& operator=(const RbfRange&) = delete;
};

struct rbf_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    rbf_options opt{};
    int sm_count = 0;
    char err[512] = {0};
    void* ws = nullptr;          // growable workspace
    size_t ws_bytes = 0;
    rbf_dev_state* d_state = nullptr;
    rbf_dev_state* h_state = nullptr;  // pinned mirror
    cudaEvent_t ev[2] = {nullptr, nullptr};
    rbf_timings tim{};
    // counters
    int64_t launches = 0;
    static constexpr int PMAX = 8192;
    static constexpr int PKINDS = 3;  // 0: A x, 1: A^T x, 2: reorthogonalization (half-step) kernels
    cudaEvent_t* pev = nullptr;   // [PKINDS][PMAX][2] start/stop events
    int pcount[PKINDS] = {0, 0, 0};     // recorded pairs per kind
    int64_t ptotal[PKINDS] = {0, 0, 0}; // launches per kind
    void* batch_state = nullptr;  // batched GKB: tuning choice, captured graph, stream
    cudaEvent_t pbase = nullptr;  // origin of the product-launch intervals since the last reset
    bool pbase_set = false;
    // Lanes: child contexts with their own stream, device state and workspace on
    // which rbf_gkb_many / rbf_hkt_many run independent problems concurrently.
    // A lane records its product timings into its owner's counters.
    static constexpr int MAX_LANES = 8;
    rbf_ctx* lane[MAX_LANES] = {};
    int lane_count = 1;              // lanes in use by the current multi-run call
    rbf_ctx* owner = nullptr;        // set on a lane: the context it belongs to
    bool own_stream = false;         // a lane owns (and destroys) its stream
    cudaEvent_t sync_ev = nullptr;   // fork (owner) or join (lane) event, no timing
    rbf_dev_state* h_many = nullptr; // pinned copies of the device state, one per run
    int h_many_cap = 0;
};
void rbf_batch_state_free(rbf_ctx* ctx);
cudaStream_t rbf_batch_stream(rbf_ctx* ctx);  // the batched driver's stream, or null
// Wait for everything the context has enqueued: its stream, its lanes' streams
// and the batched driver's stream.
rbf_status rbf_sync_all(rbf_ctx* ctx);
// Lane i of ctx (created on first use).  Errors: RBF_ERR_CUDA.
rbf_status rbf_lane(rbf_ctx* ctx, int i, rbf_ctx** out);
// Pinned host slots for `count` device-state copies.
rbf_status rbf_many_slots(rbf_ctx* ctx, int count);
// Order every lane in [0, lanes) after the work enqueued so far on ctx->stream
// (fork) and ctx->stream after everything enqueued on those lanes (join); the
// lanes' kernel-launch counts are added to ctx's.
rbf_status rbf_lanes_fork(rbf_ctx* ctx, int lanes);
rbf_status rbf_lanes_join(rbf_ctx* ctx, int lanes);

// ---- error helpers ---------------------------------------------------------
rbf_status rbf_fail(rbf_ctx* ctx, rbf_status st, const char* fmt, ...);

// Bounds-checked build: the line of the first failed index check of each
// instrumented translation unit (0 = none; always 0 in the normal build), and
// their collection into RBF_ERR_INTERNAL (call after the work has completed).
unsigned rbf_check_take_ctx();
unsigned rbf_check_take_gemv();
unsigned rbf_check_take_gkb();
unsigned rbf_check_take_batch();
unsigned rbf_check_take_select();
unsigned rbf_check_take_assemble();
unsigned rbf_check_take_mf();
unsigned rbf_check_take_fx();
rbf_status rbf_check_all(rbf_ctx* ctx);

#define RBF_CUDA(ctx, call)                                                             \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return rbf_fail((ctx), RBF_ERR_CUDA, "%s failed: %s (%s:%d)", #call,        \
                            cudaGetErrorString(e_), __FILE__, __LINE__);                \
    } while (0)

#define RBF_LAUNCHED(ctx, name)                                                         \
    do {                                                                                \
        (ctx)->launches++;                                                              \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess)                                                          \
            return rbf_fail((ctx), RBF_ERR_CUDA, "launch of %s failed: %s", name,       \
                            cudaGetErrorString(e_));                                    \
    } while (0)

#define RBF_TRY(expr)                      \
    do {                                   \
        rbf_status s_ = (expr);            \
        if (s_ != RBF_OK) return s_;       \
    } while (0)

// Grow the workspace to at least `bytes` (synchronises the stream when it
// reallocates).  Returns RBF_ERR_OOM on failure or when above the cap.
rbf_status rbf_ws_reserve(rbf_ctx* ctx, size_t bytes);

// Simple bump allocator over the workspace (256-byte aligned slices).
struct WsCarve {
    char* base;
    size_t off;
    explicit WsCarve(void* b) : base((char*)b), off(0) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base + off);
        off += count * sizeof(T);
        return p;
    }
};
inline size_t ws_align(size_t b) { return (b + 255) & ~(size_t)255; }

// ---- timing ------------------------------------------------------------------
// Launch timing (opt.timing bit 1) of kind 0 (A x), 1 (A^T x) or 2 (half-step
// kernels), recorded on `s` (default: the context stream): returns the slot or -1.
int rbf_prod_begin(rbf_ctx* ctx, int kind, cudaStream_t s = nullptr);
void rbf_prod_end(rbf_ctx* ctx, int kind, int slot, cudaStream_t s = nullptr);
void rbf_timer_start(rbf_ctx* ctx);
double rbf_timer_stop(rbf_ctx* ctx);  // ms, synchronises when timing is on

// ---- launchers (one per translation unit family) ------------------------------
// assemble.cu
rbf_status launch_assemble(rbf_ctx* ctx, const rbf_operator* op);
// Two FP64 assembled operators on the same nodes, n_interior, c and form (k may
// differ) into distinct matrices, in one pass; entries bitwise equal to two
// launch_assemble calls.
bool assemble_pairable(const rbf_operator* a, const rbf_operator* b);
rbf_status launch_assemble_pair(rbf_ctx* ctx, const rbf_operator* a, const rbf_operator* b);
rbf_status launch_evaluate(rbf_ctx* ctx, const rbf_operator* op, const double* coef,
                           const double* pts, int64_t m, double* u);
// gemv.cu
size_t gemv_ws_bytes(const rbf_ctx* ctx, int64_t n);
int gemv_t_chunks(const rbf_ctx* ctx, const rbf_operator* op);
int gemv_n_chunks(const rbf_ctx* ctx, const rbf_operator* op);  // partials of A x (FP64: column segments)
rbf_status launch_to_f32(rbf_ctx* ctx, int64_t n, const double* x, float* y, cudaStream_t s = nullptr);
// Partials of A x (column segments [gemv_n_chunks][n]) and of A^T x (row
// chunks [gemv_t_chunks][n]); FP64 x for FP64 operators, x32 for FP32 ones.
rbf_status launch_gemv_n(rbf_ctx* ctx, const rbf_operator* op, const double* x, const float* x32, double* part,
                         const int* done);
rbf_status launch_gemv_t_partial(rbf_ctx* ctx, const rbf_operator* op, const double* x,
                                 const float* x32, double* part, const int* done);
rbf_status launch_reduce_partials(rbf_ctx* ctx, int64_t n, int chunks, const double* part, double* y);
// Flat split of an n x n matrix over at most Wmax warps (flat_bound): the warps
// used and the most pieces a row is split into (at most 8).
void flat_split_plan(int64_t n, int64_t Wmax, int64_t* W, int* chunks);
// Column panels x row chunks of the A^T x kernels (vec columns per thread).
void plan_t(const rbf_ctx* ctx, int64_t n, int vec, int* panel_cols, int* panels, int* chunks);
// fx.cu: the FP64 assembled GKB products in exact integer fixed point, from two
// int64 copies of A (row-scaled NR for A z, column-scaled NC for A^T w) made
// once per GKB run, and the largest exponent field of each row / column.
struct FxCopies {
    long long* NR = nullptr;
    long long* NC = nullptr;
    int* rowE = nullptr;
    int* colE = nullptr;
};
bool fx_eligible(const rbf_ctx* ctx, const rbf_operator* op);
size_t fx_ws_bytes(const rbf_operator* op);
FxCopies fx_carve(WsCarve& wc, const rbf_operator* op);
int fx_n_chunks(const rbf_ctx* ctx, int64_t n);  // partial rows of the fixed-point A z (<= 8)
rbf_status launch_fx_prepare(rbf_ctx* ctx, const rbf_operator* op, const FxCopies& f);
rbf_status launch_fx_n(rbf_ctx* ctx, const rbf_operator* op, const FxCopies& f, const double* x, double* part,
                       const int* done);
rbf_status launch_fx_t(rbf_ctx* ctx, const rbf_operator* op, const FxCopies& f, const double* x, double* part,
                       const int* done);
// mf.cu (matrix-free products, FP32 or FP64; partial sums over `mf_chunks` centre chunks)
// Partial rows the consumer sums (mf_chunks) and rows the product writes
// (mf_part_rows >= mf_chunks; the FP32 tile-pair product folds its slots).
int mf_chunks(const rbf_ctx* ctx, const rbf_operator* op);
int mf_part_rows(const rbf_ctx* ctx, const rbf_operator* op);
// FP32 matrix-free products whose partial slots are the FP32 runs themselves
// (unscaled floats, added by the consumer with a compensated FP32 sum and
// multiplied by the form's scale): every FP32 matrix-free plan without a fold.
bool mf_slots_f32(const rbf_ctx* ctx, const rbf_operator* op);
rbf_status launch_reduce_slots_f32(rbf_ctx* ctx, int64_t n, int chunks, const float* part, double scale, double* y);
size_t mf_ws_bytes(const rbf_ctx* ctx, int64_t n);
// x: FP64 input (FP64 operators); x32 and X32 (the node coordinates, SoA
// [3][n], rounded to FP32): inputs of FP32 operators.
rbf_status launch_mf_partial(rbf_ctx* ctx, const rbf_operator* op, int trans, const double* x,
                             const float* x32, const float* X32, double* part, const int* done);  // x (FP64 op) or x32
// gkb.cu
rbf_status gkb_run(rbf_ctx* ctx, const rbf_operator* op, const double* f, int j_begin, int j_end,
                   rbf_gkb_state* st);
size_t gkb_ws_bytes(const rbf_ctx* ctx, int64_t n, int steps, int precision);
// svd.cu: batched projected problem (blockIdx.y / blockIdx.x = instance b; buffers
// strided by the capacity L: alpha [B][L], beta [B][L+1], sigma [B][L],
// ftil [B][L+1], V [B][L][ldv]); l per instance from l_arr (device) or l.
struct ProjDims {
    int B;
    int L;
    int l;
    const int* l_arr;
};
size_t svd_ws_bytes(int l);
size_t svd_ws_bytes_batch(int L, int B);
rbf_status launch_projected_svd_batch(rbf_ctx* ctx, ProjDims d, const double* alpha, const double* beta,
                                      double* sigma, double* ftil, double* V, int64_t ldv, void* ws,
                                      double* sigma1_out, double* ftil_last_out, double* U = nullptr,
                                      int64_t ldu = 0);
rbf_status launch_projected_svd(rbf_ctx* ctx, const double* alpha, const double* beta, int l,
                                double* sigma, double* ftil, double* V, int64_t ldv, void* ws);
// select.cu
struct LiftDims {           // lift coef = Z y per instance
    const int64_t* n_arr;   // device [B] sizes (batched) or null
    const int64_t* zoff;    // device [B] offsets of Z_b (batched, ld = n_b) or null
    const int64_t* coff;    // device [B] offsets of coef_b or null
    int64_t n;              // single instance: n
    int64_t ldz;            // single instance: ld of Z
    int64_t nmax;           // max n (grid size)
};
size_t select_ws_bytes(const rbf_ctx* ctx, int l);
// Single-instance HKT (rule incl. RBF_FIXED_T) on the first st->steps_done
// steps; d_coef may be NULL (no lift: only *info, with eta and rho).
rbf_status hkt_single(rbf_ctx* ctx, const rbf_gkb_state* st, int rule, double lambda_in, double* d_coef,
                      rbf_solve_info* info, double* d_curve = nullptr);
size_t select_ws_bytes_batch(const rbf_ctx* ctx, int L, int B);
// method 0: HKT with `rule`; 1: Ine-TSVD with `rank` (0 = GCV).  rule_arr /
// lam_arr (device [B], optional) give each instance its own HKT rule and
// lambda_in.
rbf_status launch_select_batch(rbf_ctx* ctx, ProjDims d, int method, int rule, double lambda_in, int rank,
                               const double* alpha, const double* beta, const double* Z, LiftDims ld,
                               double* coef, double* curve, void* ws, double* lam_out, int* idx_out,
                               int* rank_out, bool single, const int* rule_arr = nullptr,
                               const double* lam_arr = nullptr);

// mlp.cu: stop features of B batch instances after j steps (alpha [B][L],
// beta [B][L+1], sigma [B][L] from the batched projected SVD at l = d_l[b]);
// feat [B][20], NaN rows for instances with fewer than j steps.
rbf_status launch_stop_features_batch(rbf_ctx* ctx, const double* alpha, const double* beta, const double* sigma,
                                      int L, const int* d_l, int B, int j, const float* mean, const float* stdv,
                                      float* feat);
