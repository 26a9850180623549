/*
 * rbfkr.h -- C ABI of the GB300 (sm_103a) Krylov-regularization library for
 * multiquadric (MQ) RBF Kansa collocation of the 3D Helmholtz equation.
 *
 * What it computes (arXiv 2511.09798):
 *   - the Kansa collocation matrix A = [H; R] with MQ basis Phi(r) =
 *     sqrt(r^2 + c^2): interior rows L Phi = Delta Phi + k^2 Phi, Dirichlet rows
 *     Phi (Sec. 2.1, eqs. MQ, Lphi, H_entries, augmented_system);
 *   - Golub-Kahan bidiagonalization with full reorthogonalization
 *     (Algorithm 1, Sec. 3.1);
 *   - the projected SVD C_l = U~ S~ V~^T, projected GCV / L-curve choice of
 *     lambda, Hybrid Krylov-Tikhonov (Algorithm 4) and inexpensive TSVD
 *     (Algorithm 2), lifted to coefficients alpha = Z_l y;
 *   - reconstruction u(X) = sum_j alpha_j Phi(|X - X_j|) (eq. u_reconstruction).
 *
 * Conventions (all entry points):
 *   - Every pointer named d_* is DEVICE memory owned by the caller, on the
 *     device the context was created for.  The library owns only the internal
 *     workspace it allocates inside the context (see rbf_workspace_bytes).
 *   - Node coordinates are FP64 structure-of-arrays [3][n]: x[0..n), then
 *     y[0..n), then z[0..n); interior (PDE) nodes first, boundary (Dirichlet)
 *     nodes last.  Centres and collocation points coincide.
 *   - Dense matrices are row-major with a leading dimension (lda >= n).
 *     Krylov bases are column-major (each basis vector contiguous, ld >= n).
 *   - Work is enqueued on the stream given to rbf_create.  Calls that return a
 *     host scalar (steps done, lambda, rank) synchronise that stream; the
 *     others do not.
 *   - Errors are return codes; nothing throws across the ABI.  The message of
 *     the last failure is available from rbf_last_error.  Asynchronous CUDA
 *     errors surface at the next synchronising call as RBF_ERR_CUDA.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef RBFKR_H
#define RBFKR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RBF_OK = 0,
    RBF_ERR_INVALID = 1,     /* bad argument (size, pointer, parameter range) */
    RBF_ERR_OOM = 2,         /* workspace allocation failed or exceeds the cap */
    RBF_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    RBF_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    RBF_ERR_UNSUPPORTED = 5, /* combination not implemented */
    RBF_ERR_INTERNAL = 6     /* device-side consistency check failed */
} rbf_status;

typedef enum {
    RBF_FP64 = 0,  /* every step in IEEE FP64 */
    RBF_MIXED = 1  /* matrix entries and A*x / A^T*y in FP32 (partial sums of
                      short FP32 runs combined in FP64); reorthogonalization,
                      norms, alpha/beta, projected SVD and GCV in FP64 */
} rbf_precision;

typedef enum {
    RBF_ASSEMBLED = 0,   /* A stored densely (caller-owned buffer) */
    RBF_MATRIX_FREE = 1  /* entries regenerated from node coordinates per product
                            (in FP32 for RBF_MIXED, in FP64 for RBF_FP64) */
} rbf_storage;

typedef enum {
    RBF_GCV = 0,     /* argmin of the projected GCV on the lambda grid (eq. gcv_proj) */
    RBF_LCURVE = 1,  /* max discrete curvature of (ln rho_l, ln eta_l) on the grid */
    RBF_FIXED = 2,   /* lambda supplied by the caller */
    RBF_FIXED_T = 3  /* lambda = s~_1 10^t with t = lambda_in supplied by the caller */
} rbf_rule;

typedef enum {
    RBF_FORM_C = 0,   /* Phi(r) = sqrt(r^2 + c^2) */
    RBF_FORM_EPS = 1  /* phi(r; eps) = sqrt(1 + eps^2 r^2), eps = 1/c (eq. MQ): entries / c */
} rbf_form;

typedef struct rbf_ctx rbf_ctx;

/* Options fixed at context creation.  Zero-initialised fields take defaults. */
typedef struct {
    int grid_j;              /* lambda grid points J (default 321; 1 and 2 are rejected) */
    double grid_t_lo;        /* grid: lambda = s~_1 * 10^t, t in [t_lo, t_hi] (default -16) */
    double grid_t_hi;        /* (default 0; used only when t_lo < t_hi) */
    double breakdown_factor; /* tau = factor * N * eps * c_hat (default 64) */
    double cluster_tol;      /* relative gap under which Ritz values are treated
                                as a cluster in the projected SVD (default 1e-3) */
    int64_t workspace_cap;   /* max workspace bytes, 0 = unlimited */
    int timing;              /* bit 0: per-phase CUDA-event timings (synchronises at
                                each phase end); bit 1: time every GKB product launch
                                with CUDA events, no synchronisation (rbf_counters) */
    int svd_method;          /* full SVD: 0 Householder bidiagonalization + tridiagonal
                                SVD (default), 1 one-sided Jacobi */
    int64_t wait_budget;     /* polls a device-side wait (grid barrier) makes before it
                                gives up: the run stops and the call returns
                                RBF_ERR_TIMEOUT instead of waiting for ever (default
                                2^23, several seconds; a tiny value forces the timeout
                                path, which leaves the context usable) */
    int fma_products;        /* FP64 assembled operators, n <= 16384: GKB (and LSQR on
                                its state) computes A z and A^T w in exact integer
                                fixed point from two int64 copies of A made at the
                                start of each run (2 x 8 n lda bytes more workspace).
                                Sums are exact; every value is rounded at 2^-62 of the
                                largest in its row / column / vector (exact for values
                                within 2^9 of it), then one FP64 rounding per partial:
                                error <~ 2^-61 (max|A_ij| |w|_1 + |A_.j|_1 max|w_i|) per
                                output, below FP64 FMAs' for matrices like the
                                collocation matrices, normwise rather than componentwise
                                for rows / columns scaled over many orders of magnitude;
                                not bound by the FP64 pipe.  1: FP64 FMAs on A itself
                                instead.  Without room for the copies (the workspace cap
                                or device memory) the FMA products run. */
} rbf_options;

/* Operator description; filled by rbf_operator_init. */
typedef struct {
    const double* d_nodes; /* device FP64 SoA [3][n] */
    int64_t n;             /* number of nodes (= rows = columns of A) */
    int64_t n_interior;    /* rows [0, n_interior) are PDE rows, the rest Dirichlet */
    double c;              /* MQ shape parameter (c-form) */
    double k;              /* wavenumber */
    int storage;           /* rbf_storage */
    int precision;         /* rbf_precision */
    int form;              /* rbf_form */
    void* d_A;             /* device, caller-owned: double (FP64) or float (MIXED),
                              row-major n x lda; NULL for RBF_MATRIX_FREE */
    int64_t lda;           /* leading dimension in elements; even (FP64) or a
                              multiple of 4 (FP32); d_A 16-byte aligned */
} rbf_operator;

/* Golub-Kahan state.  The caller owns W, Z, alpha, beta (device).  The
 * scalar fields steps_done / breakdown / c_hat are written by rbf_gkb and
 * rbf_gkb_resume when they return. */
typedef struct {
    double* d_W;      /* n x (capacity+1), column-major, ld = ldw: w_1 .. w_{l+1} */
    int64_t ldw;
    double* d_Z;      /* n x capacity, column-major, ld = ldz: z_1 .. z_l */
    int64_t ldz;
    double* d_alpha;  /* [capacity]:   d_alpha[j-1] = alpha_j */
    double* d_beta;   /* [capacity+1]: d_beta[j-1]  = beta_j (beta_1 = |f|) */
    int capacity;     /* maximum number of steps the buffers hold */
    int64_t n;
    int steps_done;   /* l: completed steps */
    int breakdown;    /* 0 none; 1 alpha_j <= tau (l = j-1); 2 beta_{j+1} <= tau (l = j,
                         beta_{l+1} = 0, w_{l+1} = 0); 3 a norm was not finite (NaN or
                         Inf in f, the nodes or the operator): the run stops as for 1
                         (alpha_j) or 2 (beta_{j+1}), l counts the steps before it */
    double c_hat;     /* running estimate of |A|_2 used by the breakdown test */
} rbf_gkb_state;

/* Host-side results of a regularized solve. */
typedef struct {
    double lambda;   /* lambda used (HKT) */
    int index;       /* grid index of lambda (-1 for RBF_FIXED) */
    int rank;        /* truncation rank (Ine-TSVD) */
    int steps;       /* l, the projected dimension used */
    double sigma1;   /* largest Ritz value s~_1 */
    double eta;      /* |y| = |alpha| (Z_l has orthonormal columns), eq. eta_proj */
    double rho;      /* projected residual |C_l y - beta_1 e_1|, eq. rho_proj */
} rbf_solve_info;

/* Per-phase device time of the last calls, milliseconds (timing option). */
typedef struct {
    double assemble_ms;
    double gkb_ms;
    double svd_ms;
    double select_ms;  /* GCV / L-curve / rank choice and projected solve */
    double lift_ms;
    double evaluate_ms;
    int gkb_steps;
} rbf_timings;

/* Counters since creation or the last reset: kernel launches made by the
 * library, and (when bit 1 of opt.timing is set) the device time of the GKB
 * matrix-vector product launches (index 0: p = A z, index 1: r = A^T w) and of
 * the half-step (reorthogonalization) kernels, measured with CUDA events
 * recorded around each launch on the stream it is launched on.  With this bit
 * set the batched GKB launches its step loop directly instead of replaying a
 * captured graph, so that every launch can be timed. */
typedef struct {
    int64_t launches;           /* every kernel launch issued by the library */
    int64_t product_launches[2];/* timed product launches (A, A^T) */
    double product_ms[2];       /* their summed device time, milliseconds */
    double product_busy_ms;     /* length of the union of those launch intervals: the time
                                   during which at least one product ran (equal to the sum
                                   when products never overlap; smaller when products of
                                   concurrent runs, rbf_gkb_many, overlap) */
    int64_t reorth_launches;    /* timed half-step (reorthogonalization) kernel launches */
    double reorth_ms;           /* their summed device time, milliseconds */
} rbf_counters;

/* ---- context --------------------------------------------------------- */

/* Create a context on `device` enqueuing on `cuda_stream` (a cudaStream_t, or
 * NULL for the legacy default stream).  `opt` may be NULL (defaults).
 * Errors: RBF_ERR_INVALID (ctx NULL, opt->grid_j 1 or 2), RBF_ERR_CUDA (device
 * unusable). */
rbf_status rbf_create(rbf_ctx** ctx, int device, void* cuda_stream, const rbf_options* opt);

/* Release the context and its workspace.  NULL is accepted. */
rbf_status rbf_destroy(rbf_ctx* ctx);

/* Message of the last failing call on this context ("" if none). */
const char* rbf_last_error(const rbf_ctx* ctx);

/* Upper bound of the internal workspace bytes for a GKB of `steps` steps plus
 * the projected solve, for an operator of size n (FP64 assembled, unless
 * opt.fma_products: with the two fixed-point copies of A, lda = n rounded up
 * to even). */
size_t rbf_workspace_bytes(const rbf_ctx* ctx, int64_t n, int steps, int storage, int precision);

/* Timings of the most recent calls (zeros unless opt.timing was set). */
rbf_status rbf_get_timings(const rbf_ctx* ctx, rbf_timings* out);

/* Read the counters (synchronises the stream when product timing is on) and
 * reset them to zero when `reset` is non-zero.  Product timing keeps at most
 * 8192 launches per reset; later launches are counted but not timed. */
rbf_status rbf_get_counters(rbf_ctx* ctx, rbf_counters* out, int reset);

/* ---- operator ------------------------------------------------------- */

/* Fill *op after validating the arguments (Sec. 2.1: centres = collocation
 * points, interior rows first).  No device work.  Errors: RBF_ERR_INVALID for
 * n <= 0, n_interior outside [0, n], c <= 0, k < 0, d_nodes NULL, an assembled
 * operator without d_A, lda < n or misaligned, unknown enum values. */
rbf_status rbf_operator_init(rbf_ctx* ctx, rbf_operator* op, const double* d_nodes, int64_t n,
                             int64_t n_interior, double c, double k, int storage, int precision,
                             int form, void* d_A, int64_t lda);

/* Fill the caller's d_A with the collocation matrix (eqs. H_entries,
 * augmented_system): FP64 or FP32 entries by op->precision.  Assembled
 * operators only (RBF_ERR_INVALID otherwise). */
rbf_status rbf_assemble(rbf_ctx* ctx, const rbf_operator* op);

/* d_y = A d_x (trans = 0) or d_y = A^T d_x (trans = 1), FP64 vectors of length
 * n; the product runs in the operator's precision and storage (the matrix-vector
 * product of Algorithm 1, steps r = A^T w and p = A z). */
rbf_status rbf_matvec(rbf_ctx* ctx, const rbf_operator* op, int trans, const double* d_x, double* d_y);

/* ---- Golub-Kahan bidiagonalization (Algorithm 1) --------------------- */

/* Run `steps` steps from beta_1 = |f|, w_1 = f / beta_1 into *st (capacity >=
 * steps, buffers sized for n = op->n).  Full reorthogonalization of r against
 * z_1..z_{j-1} before alpha_j and of p against w_1..w_j before beta_{j+1}
 * (classical Gram-Schmidt applied twice).  Stops early on breakdown (tau =
 * factor * N * eps * c_hat).  Synchronises the stream to return steps_done. */
rbf_status rbf_gkb(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int steps,
                   rbf_gkb_state* st);

/* Continue a state produced by rbf_gkb for `more_steps` further steps (same
 * operator); a state that already broke down is returned unchanged. */
rbf_status rbf_gkb_resume(rbf_ctx* ctx, const rbf_operator* op, rbf_gkb_state* st, int more_steps);

/* Checkpoint of a GKB state in host memory: copies w_1..w_{l+1} into h_W
 * (n x (l+1), column-major, ld n), z_1..z_l into h_Z (n x l), alpha_1..alpha_l
 * and beta_1..beta_{l+1}, with l = st->steps_done (0 <= l <= capacity); the
 * scalars steps_done, breakdown and c_hat stay in *st for the caller to keep.
 * Synchronises.  RBF_ERR_INVALID for NULL pointers or an inconsistent state. */
rbf_status rbf_gkb_snapshot(rbf_ctx* ctx, const rbf_gkb_state* st, double* h_W, double* h_Z, double* h_alpha,
                            double* h_beta);

/* Restore a checkpoint written by rbf_gkb_snapshot into the device buffers of
 * *st (capacity >= steps_done >= 1, the same n) and set its scalars, so that
 * rbf_gkb_resume continues exactly as the run it was taken from would have.
 * Synchronises (the host arrays may be released on return).
 * RBF_ERR_INVALID for NULL pointers or values out of range. */
rbf_status rbf_gkb_restore(rbf_ctx* ctx, rbf_gkb_state* st, const double* h_W, const double* h_Z,
                           const double* h_alpha, const double* h_beta, int steps_done, int breakdown, double c_hat);

/* Several independent GKB runs at once (Algorithm 1 for each): run i applies
 * ops[i] to d_f[i] for `steps` steps into states[i], exactly as rbf_gkb would
 * (same kernels, so each run's results are bitwise those of rbf_gkb).  The
 * runs are spread over `lanes` child streams of the context (at most 8; 0 =
 * one lane per run up to 8; reduced when the half-step kernels of that many
 * runs would not fit on the SMs together), run i on lane i mod lanes, enqueued one GKB
 * step per lane in turn, so that one run's latency-bound reorthogonalization
 * kernels overlap another run's matrix-vector products.  Each lane owns its
 * own workspace (opt.workspace_cap applies per lane) and device state.  With
 * `assemble` non-zero each assembled operator is first filled (rbf_assemble;
 * FP64 operators that differ only in k are assembled two at a time, sharing
 * the distances, with the same entries), so runs must then not share a matrix
 * buffer.  The lanes
 * start after the work already enqueued on the context stream, and the
 * context stream waits for all of them before later work.  Synchronises once;
 * fills every state's steps_done, breakdown and c_hat.  Errors as rbf_gkb,
 * for the first failing run. */
rbf_status rbf_gkb_many(rbf_ctx* ctx, int count, const rbf_operator* ops, const double* const* d_f, int steps,
                        rbf_gkb_state* states, int lanes, int assemble);

/* ---- projected problem (Algorithms 2 and 4) -------------------------- */

/* SVD of the (l+1) x l lower bidiagonal C_l of *st (l = st->steps_done):
 * d_sigma[l] (descending), d_ftil[l+1] = U~^T (beta_1 e_1), d_V (l x l,
 * column-major, ld = ldv >= l, columns v~_i).  FP64. */
rbf_status rbf_projected_svd(rbf_ctx* ctx, const rbf_gkb_state* st, double* d_sigma, double* d_ftil,
                             double* d_V, int64_t ldv);

/* Hybrid Krylov-Tikhonov (Algorithm 4): choose lambda by `rule` on the grid
 * lambda = s~_1 10^t (or take lambda_in for RBF_FIXED, or s~_1 10^lambda_in
 * for RBF_FIXED_T), solve the projected Tikhonov problem and lift: d_coef[n] =
 * Z_l y_lambda.  d_curve (optional, length J) receives GCV_l on the grid
 * (RBF_GCV) or the curvature (RBF_LCURVE, end points = -inf).  Synchronises;
 * fills *info (eta and rho at the chosen lambda). */
rbf_status rbf_hkt(rbf_ctx* ctx, const rbf_gkb_state* st, int rule, double lambda_in,
                   double* d_coef, double* d_curve, rbf_solve_info* info);

/* rbf_hkt for `count` finished states at once (same rule and lambda_in for all,
 * no GCV curve output): d_coef[i] receives Z_l y_lambda of states[i], infos[i]
 * (optional) its solve information.  Spread over `lanes` child streams as in
 * rbf_gkb_many; synchronises once; results are bitwise those of rbf_hkt. */
rbf_status rbf_hkt_many(rbf_ctx* ctx, int count, const rbf_gkb_state* states, int rule, double lambda_in,
                        double* const* d_coef, rbf_solve_info* infos, int lanes);

/* Inexpensive TSVD (Algorithm 2): rank by GCV_l(k) when rank == 0, else the
 * given rank (1..l); d_coef[n] = Z_l V~_k S~_k^{-1} f~_{1:k}.  d_curve
 * (optional, length l) receives GCV_l(k).  Synchronises; fills *info. */
rbf_status rbf_ine_tsvd(rbf_ctx* ctx, const rbf_gkb_state* st, int rank, double* d_coef,
                        double* d_curve, rbf_solve_info* info);

/* LSQR as iterative regularization (Sec. 3.4) on a finished GKB run: the k-th
 * iterate x_k = Z_k y_k, y_k the least-squares solution of C_k y = beta_1 e_1,
 * with k chosen from the sequence (rho_k, eta_k) = (|A x_k - f|, |x_k|),
 * k = 1..l: RBF_LCURVE = the corner (maximum signed curvature of
 * (ln rho_k, ln eta_k) by central differences along decreasing k, stationary
 * points excluded), RBF_GCV = argmin rho_k^2 / ((l+1) - k)^2, RBF_FIXED =
 * k_fixed (1..l).  d_coef[n] = x_k; d_curve (optional, length l) receives the
 * rule's values.  l <= 511.  Synchronises; info->rank = k, eta and rho at k. */
rbf_status rbf_lsqr(rbf_ctx* ctx, const rbf_gkb_state* st, int rule, int k_fixed, double* d_coef,
                    double* d_curve, rbf_solve_info* info);

/* Full SVD of an assembled FP64 operator (Algorithm 3 step 1), 2 <= n <=
 * 8192, by Householder bidiagonalization and the tridiagonal SVD of the
 * bidiagonal (opt.svd_method 0) or one-sided Jacobi (1; *sweeps = number of
 * sweeps, 0 for the first method): d_sigma[n] receives the singular values in
 * descending order; with d_f given, d_fhat[n] receives f^ = U^T f; d_V
 * (optional, n x n column-major) the right singular vectors in the same order.
 * Workspace: about 3 n^2 doubles plus 8 n^2 (bidiagonal path) or 2 n^2
 * (Jacobi).  Synchronises.  RBF_ERR_UNSUPPORTED for other operators. */
rbf_status rbf_svd_full(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, double* d_sigma,
                        double* d_fhat, double* d_V, int* sweeps);

/* Full-SVD Tikhonov (Algorithm 3): lambda by GCV on the grid lambda = s_1 10^t
 * (eq. gcv_svd, denominator (N - r) + sum_{i<=r} (1 - phi_i), numerical rank
 * r = #{s_i > N eps s_1}, s_perp = sum_{i>r} f^_i^2) or fixed (RBF_FIXED);
 * d_coef[n] = sum_{i<=r} phi_i / s_i f^_i v_i (eq. tikh_svd_solution).
 * Assembled FP64 operators, n <= 8192.  Synchronises; info: lambda, index,
 * rank = r, steps = Jacobi sweeps (0 on the bidiagonal path), sigma1. */
rbf_status rbf_tikhonov(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int rule,
                        double lambda_in, double* d_coef, rbf_solve_info* info);

/* Full TSVD (eq. tsvd_solution): d_coef[n] = sum_{i<=k} f^_i / s_i v_i with
 * k = rank (1..n) or, for rank = 0, the GCV choice over k = 1..min(r, N-1):
 * GCV(k) = (sum_{k<i<=r} f^_i^2 + s_perp) / (N - k)^2.  Same operators and
 * synchronisation as rbf_tikhonov; info->rank = k. */
rbf_status rbf_tsvd(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, int rank, double* d_coef,
                    rbf_solve_info* info);

/* ---- reconstruction (eq. u_reconstruction) --------------------------- */

/* d_u[m] = sum_j d_coef[j] Phi(|P_t - X_j|) at the m points d_points (FP64 SoA
 * [3][m]).  Always FP64 (also for RBF_MIXED operators): the coefficients of an
 * ill-conditioned collocation system cancel, so FP32 basis values would lose
 * the reconstruction.  Uses the operator's form (c or eps). */
rbf_status rbf_evaluate(rbf_ctx* ctx, const rbf_operator* op, const double* d_coef,
                        const double* d_points, int64_t m, double* d_u);

/* ---- batched instances (many uneven problems in one graph launch) ------ */

/* A batch of independent collocation problems of uneven size, advanced through
 * GKB together.  Concatenated layouts use off_b = sum_{a<b} n_a. */
typedef struct {
    int count;                   /* number of instances B >= 1 */
    const int64_t* n;            /* host [B] nodes per instance */
    const int64_t* n_interior;   /* host [B] PDE rows per instance */
    const double* c;             /* host [B] MQ shape parameters */
    const double* k;             /* host [B] wavenumbers */
    const double* d_nodes;       /* device FP64: instance b's SoA [3][n_b] at 3 * off_b */
    const double* d_f;           /* device FP64: f_b at off_b */
    int capacity;                /* L: maximum GKB steps per instance */
    double* d_W;                 /* device: W_b (n_b x (L+1), column-major, ld n_b) at (L+1) * off_b */
    double* d_Z;                 /* device: Z_b (n_b x L, ld n_b) at L * off_b */
    double* d_alpha;             /* device [B][L] */
    double* d_beta;              /* device [B][L+1] */
    int* steps_done;             /* host [B], written by rbf_batch_gkb */
    int* breakdown;              /* host [B], written by rbf_batch_gkb (codes as rbf_gkb_state.breakdown) */
    const int* steps_limit;      /* host [B] or NULL: instance b stops after min(steps, steps_limit[b])
                                    steps (>= 1), with beta and w of the next step written as after
                                    a full run of that length */
} rbf_batch;

/* Autotuner choice for the batched matrix-free product (see rbf_batch_gkb). */
typedef struct {
    int mf_outputs_per_thread;   /* rows held in registers per lane (tile pairs of 32 x this many nodes) */
    int mf_threads;              /* threads per CTA */
    int candidates;              /* configurations timed */
    double best_ms;              /* time of one A and one A^T product of the batch, best config */
    int graph_kernels;           /* kernels in the captured step graph (0 if not captured) */
} rbf_tuning;

/* Run `steps` GKB steps (Algorithm 1, same reorthogonalization and breakdown
 * rule as rbf_gkb) on every instance of the batch, mixed precision with the
 * matrix-free FP32 product (entries regenerated from the nodes; FP64
 * reorthogonalization, norms and scalars).  All instances advance in lock
 * step: per step one batched A^T product, one cooperative reorthogonalization
 * kernel over the concatenated rows, one batched A product and one more
 * reorthogonalization kernel; the whole step loop is captured once into a CUDA
 * graph and launched as one graph.  Instances that break down stop
 * individually.  On the first call for a batch shape the product's tile shape
 * is chosen by timing candidate configurations on the batch itself (see
 * rbf_get_tuning).  Synchronises; fills steps_done and breakdown.  Errors:
 * RBF_ERR_INVALID (sizes, pointers, steps > capacity or > n_b), RBF_ERR_TIMEOUT
 * (a bounded grid barrier gave up). */
rbf_status rbf_batch_gkb(rbf_ctx* ctx, rbf_batch* batch, int steps, int form);

/* HKT (Algorithm 4) for every instance of a batch after rbf_batch_gkb: projected
 * SVD, lambda by `rule` (RBF_GCV or RBF_LCURVE) on each instance's grid, solve
 * and lift into d_coef (device, instance b at off_b).  h_lambda: host [B] out. */
rbf_status rbf_batch_hkt(rbf_ctx* ctx, const rbf_batch* batch, int rule, double* d_coef, double* h_lambda);

/* rbf_batch_hkt with a rule per instance: h_rules[b] in {RBF_GCV, RBF_LCURVE,
 * RBF_FIXED, RBF_FIXED_T} with h_lambda_in[b] its lambda (RBF_FIXED) or t
 * (RBF_FIXED_T; ignored by the grid rules).  Host arrays of length B.
 * Synchronises; h_lambda[b] receives the lambda used. */
rbf_status rbf_batch_hkt_each(rbf_ctx* ctx, const rbf_batch* batch, const int* h_rules, const double* h_lambda_in,
                              double* d_coef, double* h_lambda);

/* Reconstruction for every instance: d_u (device, instance b at moff_b =
 * sum_{a<b} m_a) at the m_b points of d_points (device FP64 SoA [3][m_b] at
 * 3 * moff_b), FP64. */
rbf_status rbf_batch_evaluate(rbf_ctx* ctx, const rbf_batch* batch, int form, const double* d_coef,
                              const double* d_points, const int64_t* m, double* d_u);

/* The autotuner's last choice. */
rbf_status rbf_get_tuning(const rbf_ctx* ctx, rbf_tuning* out);

/* ---- learned stopping index and lambda -----------------------------------
 *
 * The paper stops GKB at a fixed l and picks lambda by GCV or the L-curve
 * (Sec. 3.2-3.4); its closing discussion leaves cheaper stopping as future
 * work.  These entry points carry a small regressor that predicts, from the
 * first 10 GKB steps, the stopping index l and log10 lambda, so that GKB can
 * end early and the selection sweep is skipped.  The network is not in the
 * paper: a 20 -> 128 -> 128 -> 2 perceptron with exact (erf) GELU after both
 * hidden layers, FP32 parameters and arithmetic (gradients accumulated in
 * FP64).  Parameters are one FP32 vector of RBF_MLP_PARAMS elements laid out
 * as W1 [20][128] (row-major, input index first), b1 [128], W2 [128][128],
 * b2 [128], W3 [128][2], b3 [2]; the layer computes h_out = h_in W + b.
 * Inputs d_x are [batch][20] row-major, outputs and targets [batch][2]. */
#define RBF_MLP_IN 20
#define RBF_MLP_HIDDEN 128
#define RBF_MLP_OUT 2
#define RBF_MLP_PARAMS (20 * 128 + 128 + 128 * 128 + 128 + 128 * 2 + 2)

/* d_y = network(d_x).  Does not synchronise.  RBF_ERR_INVALID on NULL
 * pointers or batch < 1. */
rbf_status rbf_mlp_forward(rbf_ctx* ctx, const float* d_params, const float* d_x, int batch, float* d_y);

/* Gradient of the loss sum_(s,o) (y_so - t_so)^2 / (2 batch) with respect to
 * the parameters, written to d_grad (RBF_MLP_PARAMS floats, same layout as the
 * parameters; each element summed over the batch in sample order, so the
 * result is deterministic).  When h_loss is not NULL the loss is written there
 * and the stream is synchronised.  Uses the context workspace (about
 * 4 KiB per sample). */
rbf_status rbf_mlp_grad(rbf_ctx* ctx, const float* d_params, const float* d_x, const float* d_t, int batch,
                        float* d_grad, float* h_loss);

/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias correction for step
 * t >= 1) of d_params with moments d_m, d_v (RBF_MLP_PARAMS floats each,
 * zero before step 1). */
rbf_status rbf_mlp_adam(rbf_ctx* ctx, float* d_params, float* d_m, float* d_v, const float* d_grad, int t,
                        float lr);

/* rbf_mlp_grad followed by rbf_mlp_adam (d_grad receives the gradient). */
rbf_status rbf_mlp_train_step(rbf_ctx* ctx, float* d_params, float* d_m, float* d_v, int t, float lr,
                              const float* d_x, const float* d_t, int batch, float* d_grad, float* h_loss);

/* The 20 network inputs after j (1 <= j <= 10) completed GKB steps of `st`,
 * from the projected problem C_j (Sec. 3.2): log10 s~_1, log10(s~_i / s~_1)
 * for i = 2..10, and log10(rho_i / beta_1) for i = 1..10, where rho_i is the
 * least-squares residual min_y |C_i y - beta_1 e_1| after i steps.  Entries
 * past j repeat the last available value (singular values: -300); a zero
 * residual is written as -300.  When d_mean and d_std (20 floats each) are
 * given the features are standardised, (f - mean) / std.  d_feat receives 20
 * floats.  Does not synchronise.  RBF_ERR_INVALID when j is out of range or
 * the state has fewer than j steps. */
rbf_status rbf_stop_features(rbf_ctx* ctx, const rbf_gkb_state* st, int j, const float* d_mean,
                             const float* d_std, float* d_feat);

/* Reconstruction (eq. u_reconstruction) for ncoef coefficient vectors at
 * once: d_u[c][t] = sum_j d_coefs[c][j] Phi(|P_t - X_j|) (times 1/c in the
 * eps form), FP64, with d_coefs [ncoef][ldc] (ldc >= n), d_points SoA [3][m]
 * and d_u [ncoef][m].  Used to score many candidate solutions against a known
 * field (training labels for the learned stop).  Does not synchronise. */
rbf_status rbf_evaluate_many(rbf_ctx* ctx, const rbf_operator* op, const double* d_coefs, int64_t ldc,
                             int ncoef, const double* d_points, int64_t m, double* d_u);

/* Error table for labelling: for each l in h_ells (host, n_ell values, each
 * 1 <= l <= st->steps_done <= 1023) and each lambda of the context grid whose
 * index is a multiple of t_stride (Jp = (J - 1) / t_stride + 1 values,
 * lambda = s~_1(l) 10^t), the relative max-norm error
 * max_t |u_t - uref_t| / max_t |uref_t| of the HKT reconstruction u = G_l y_lambda
 * (Algorithm 4 step 9 in SVD form, eq. u_reconstruction).  d_G is column-major
 * m x l_max with ld ldg >= m, column i = Phi(P, X) z_{i+1} (rbf_evaluate_many on
 * the columns of Z); d_uref [m]; d_err receives [n_ell][Jp] doubles.
 * Synchronises. */
rbf_status rbf_hkt_error_table(rbf_ctx* ctx, const rbf_gkb_state* st, const double* d_G, int64_t ldg,
                               int64_t m, const double* d_uref, int n_ell, const int* h_ells, int t_stride,
                               double* d_err);

/* A trained stop network and the rules around it (all host fields). */
typedef struct {
    const float* d_params;     /* RBF_MLP_PARAMS floats (device) */
    const float* d_feat_mean;  /* 20 floats (device) or NULL: feature standardisation */
    const float* d_feat_std;   /* 20 floats (device) or NULL */
    float out_mean[2];         /* outputs are standardised ln l and t = log10(lambda / s~_1): */
    float out_std[2];          /*   value = output * out_std + out_mean */
    int feat_steps;            /* GKB steps before the prediction, 1..10 */
    int l_min, l_max;          /* predicted l is clamped to [l_min, l_max]; l_max is the fallback's l */
    int window;                /* acceptance: eta at t compared with l - window steps ... */
    double accept_tol;         /* ... relative change at most accept_tol */
    double t_min, t_max;       /* acceptance: predicted t must lie in [t_min, t_max] */
    int fallback_rule;         /* RBF_GCV or RBF_LCURVE */
    double z_max;              /* acceptance: every standardised feature within [-z_max, z_max]
                                  (inputs like the training set's); 0 = no bound */
} rbf_stopnet;

/* Floats of the device buffer that rbf_stopnet_init / rbf_stopnet_load fill:
 * the parameters, then the feature mean and std (20 floats each). */
#define RBF_STOPNET_DEVICE_FLOATS (RBF_MLP_PARAMS + 2 * RBF_MLP_IN)

/* Make a stop network from host arrays: the parameters h_params
 * (RBF_MLP_PARAMS floats, layout above) and the feature standardisation
 * h_feat_mean, h_feat_std (20 floats each, or both NULL for none) are copied
 * into the caller-owned device buffer d_storage (RBF_STOPNET_DEVICE_FLOATS
 * floats), and *net is filled to point at it; h_out = {out_mean[0],
 * out_mean[1], out_std[0], out_std[1]} (std > 0), h_rules = {l_min, l_max,
 * window, fallback_rule} (10 <= l_min <= l_max <= 1023; RBF_GCV or
 * RBF_LCURVE), h_tols = {accept_tol, t_min, t_max, z_max}; feat_steps = 10.
 * Synchronises (the host arrays may be released on return).  RBF_ERR_INVALID
 * for NULL arguments or rules out of range. */
rbf_status rbf_stopnet_init(rbf_ctx* ctx, rbf_stopnet* net, float* d_storage, const float* h_params,
                            const float* h_feat_mean, const float* h_feat_std, const float* h_out, const int* h_rules,
                            const double* h_tols);

/* Write *net (parameters, standardisation, output scaling, acceptance rules
 * and feat_steps) to the file `path` in the library's binary layout (magic
 * "RBFSTOP1", native little-endian; see stopnet.cu).  Synchronises.
 * RBF_ERR_INVALID when the file cannot be written. */
rbf_status rbf_stopnet_save(rbf_ctx* ctx, const rbf_stopnet* net, const char* path);

/* Read a file written by rbf_stopnet_save and initialise *net on d_storage
 * (RBF_STOPNET_DEVICE_FLOATS floats, caller-owned) as rbf_stopnet_init does.
 * RBF_ERR_INVALID for a missing file, a wrong magic or size, trailing bytes or
 * rules out of range. */
rbf_status rbf_stopnet_load(rbf_ctx* ctx, const char* path, rbf_stopnet* net, float* d_storage);

typedef struct {
    int l_pred;          /* predicted stopping index after clamping (0 when no prediction was made) */
    double t_pred;       /* predicted log10(lambda / s~_1) */
    int accepted;        /* 1: the learned (l, lambda) solution is returned; 0: fallback HKT */
    int in_distribution; /* 1: finite features within z_max of the training set */
    double eta_change;   /* |eta_l - eta_{l-window}| / eta_l at t_pred (NaN when accept_tol is inf) */
    int steps;           /* GKB steps held by the state at return */
    rbf_solve_info solve;/* the returned projected solve */
} rbf_learned_info;

/* Learned-stop HKT: GKB for net->feat_steps steps from f, the stop features,
 * one network forward, GKB resumed to the predicted l (Algorithm 1), then the
 * projected Tikhonov solve at lambda = s~_1 10^t (Algorithm 4 steps 2-10).
 * The prediction is accepted when the standardised features lie within
 * z_max, t lies in [t_min, t_max] and the solution norm eta at that t changed
 * by at most accept_tol relative over the last `window` steps (a test skipped
 * when accept_tol is +inf); otherwise GKB
 * continues to l_max and lambda comes from fallback_rule.  st must hold
 * capacity >= l_max; d_coef[n] receives Z_l y.  Synchronises; fills *info. */
rbf_status rbf_learned_hkt(rbf_ctx* ctx, const rbf_operator* op, const double* d_f, const rbf_stopnet* net,
                           rbf_gkb_state* st, double* d_coef, rbf_learned_info* info);

/* Batched learned-stop HKT: one batched GKB run of net->feat_steps steps for
 * all instances, their stop features and one network forward, then a second
 * batched run (the first steps recomputed) that stops each instance at its
 * own step count -- the predicted l when accepted (same tests as
 * rbf_learned_hkt except the eta test, which is not run), l_max otherwise --
 * and the projected solves with the predicted t or the fallback rule.  The
 * batch's steps_limit is ignored.  d_coef as rbf_batch_hkt; h_info [B]
 * receives each instance's decision (eta_change NaN; solve.lambda and
 * solve.steps filled).  Synchronises. */
rbf_status rbf_batch_learned_hkt(rbf_ctx* ctx, rbf_batch* batch, const rbf_stopnet* net, double* d_coef,
                                 rbf_learned_info* h_info);

/* ---- bounds-checked build (diagnostics, not part of the method) -------------
 *
 * The library can be built with -DRBFKR_CHECKED (librbfkr_checked.so): every
 * device index whose range follows from the host's planning (partial-sum
 * slots, shared-memory slab sizes, dot-partial and group-sum offsets, matrix
 * columns within lda) is tested before use; a failed test skips the access and
 * records the source line, and the next synchronising call (or rbf_check)
 * returns RBF_ERR_INTERNAL with the file and line in rbf_last_error.  The
 * normal build compiles the tests away. */

/* 1 for the bounds-checked build, 0 otherwise. */
int rbf_checked_build(void);

/* Wait for all work of the context (its stream, its lanes and the batched
 * driver's stream) and return RBF_ERR_INTERNAL if a device index check failed
 * since the last report (always RBF_OK in the normal build, apart from CUDA
 * errors). */
rbf_status rbf_check(rbf_ctx* ctx);

/* Enqueue one index test that fails by construction and touches no memory, so
 * that the next rbf_check of a bounds-checked build reports RBF_ERR_INTERNAL
 * (the normal build reports nothing): a test of the reporting path itself. */
rbf_status rbf_check_selftest(rbf_ctx* ctx);

/* ---- measurement (not part of the method) ------------------------------- */

/* Throughput probe of the FP64 units (the roofline peak of the FP64
 * matrix-vector products): mode 0 FP64 FMA (8 independent chains per
 * thread), 1 FP64 MMA (mma.sync m8n8k4, 4 independent accumulators per warp),
 * 2 both in every warp; `iters` iterations per thread on one resident wave of
 * CTAs.  *ms receives the CUDA-event time on the context stream, *flops the
 * floating-point operations (an FMA counts 2, an m8n8k4 MMA 512).  d_out:
 * device scratch of (SMs x 8 x 256) doubles, never written in practice.
 * Synchronises.  RBF_ERR_INVALID for other modes, iters < 1 or NULL outputs. */
rbf_status rbf_probe_fp64(rbf_ctx* ctx, int mode, long long iters, double* d_out, double* ms, double* flops);

/* ---- allocation-free product (no counterpart in the paper) ------------- */

/* Elements of the library's static device scratch used by rbf_matvec_t_noalloc
 * (8 MiB of FP64, held by every GPU that loads the library until exit). */
#define RBF_NOALLOC_SCRATCH_DOUBLES (1 << 20)

/* d_y = A^T d_x for an FP64 row-major d_A (n x lda, lda even, 16-byte aligned),
 * enqueued on `cuda_stream` (a cudaStream_t or NULL), without allocating: no
 * context is needed, and no cudaMalloc, cudaFree or allocating library routine
 * is called.  It is meant for callers that cannot allocate device memory, such
 * as code whose device memory is reserved in advance by another allocator or a
 * latency-critical loop where the device-wide synchronisation that cudaMalloc /
 * cudaFree may cause is not acceptable.  The row-chunk partial sums go to a
 * file-scope device array of RBF_NOALLOC_SCRATCH_DOUBLES doubles; n must fit
 * (the partials need at least ceil(n / 4096) chunks of n doubles, so n up to
 * about 64 000), otherwise RBF_ERR_INVALID.  The first call on a device (with
 * that device current) looks up the array's device address; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process, so no call may follow a cudaDeviceReset of that device (the reset
 * unloads the module and the array may move).  All calls share the one array
 * and every call overwrites the partials it reads, so calls that overlap on
 * the GPU (on different streams or host threads) race and must be ordered by
 * the caller.  Returns RBF_ERR_INVALID for NULL pointers or bad sizes and
 * alignment, RBF_ERR_CUDA when a CUDA call or launch fails, and also, without
 * launching anything, when an earlier CUDA error is still pending on this host
 * thread (it is left in place for its owner; no message is kept: there is no
 * context). */
rbf_status rbf_matvec_t_noalloc(const double* d_A, int64_t lda, int64_t n, const double* d_x,
                                double* d_y, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RBFKR_H */
