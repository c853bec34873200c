/*
 * vl.h -- C ABI of the GB300 iterative Vecchia-Laplace library (libvl.so).
 *
 * The library computes, for a latent Gaussian-process model with a non-Gaussian
 * likelihood (Kuendig & Sigrist, "Iterative Methods for Vecchia-Laplace
 * Approximations for Latent Gaussian Process Models"):
 *   - the Vecchia factor Sigma_tilde^{-1} = B^T D^{-1} B           (Section 2.1)
 *   - the Laplace mode b* by Newton's method                       (Eq. newton)
 *   - the negative log-marginal likelihood L^VLA with the
 *     log-determinant by stochastic Lanczos quadrature             (Eqs. VLA_loss,
 *                                                                   logdetsplit,
 *                                                                   logdetsplit2, def_SLQ)
 *   - latent predictive means and variances                        (Eq. latentpostpredictive,
 *                                                                   Algorithm simAlgo)
 * All linear solves with W + Sigma_tilde^{-1} use preconditioned CG
 * (Appendix, "PCG algorithm with Lanczos tridiagonal matrix") with the VADU, LVA
 * or LRAC preconditioner (Section 3.1). Every step runs in CUDA kernels on one
 * GPU; there is no CPU fallback.
 *
 * Conventions for every call:
 *   - Status codes are returned; nothing throws across the ABI. A message for the
 *     last failure on a context is available from vl_last_error().
 *   - Pointer arguments may be host or device memory; the library asks the CUDA
 *     driver which (cudaPointerGetAttributes) and copies host data itself. Device
 *     pointers must be on the context's device.
 *   - "caller order" is the row order of the caller's location array. The Vecchia
 *     ordering is given by `order` (order[k] = caller index of the k-th point).
 *   - Matrices of right-hand sides are n x t, row-major (t values of a point are
 *     contiguous), float64.
 *   - All work is issued on the context's stream. Calls that return host scalars
 *     synchronise that stream; the others may return before the GPU finishes,
 *     except that results written to host pointers are complete on return.
 *   - The caller owns every input and output buffer. The library owns the opaque
 *     handles. Device memory comes from the workspace given to vl_ctx_create (or
 *     from one allocation of ws_bytes made there if none is given); nothing is
 *     allocated on the device after that. Running out of it is VL_ERR_OOM.
 *   - On an error, handles stay valid and destroyable; outputs are unspecified.
 */
#ifndef VL_H_
#define VL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vl_status {
  VL_OK = 0,
  VL_ERR_INVALID_ARG = 1,   /* bad size, pointer or option                     */
  VL_ERR_OOM = 2,           /* workspace exhausted                              */
  VL_ERR_NOT_SPD = 3,       /* a Cholesky pivot <= 0 (message names the row)    */
  VL_ERR_NOT_CONVERGED = 4, /* CG or Newton hit its iteration cap               */
  VL_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up               */
  VL_ERR_CUDA = 6,          /* a CUDA runtime call failed                       */
  VL_ERR_STATE = 7          /* call made on a handle in the wrong state         */
} vl_status;

/* Covariance c(h) of the latent GP (Section 4.1 writes the Matern nu = 3/2 form). */
typedef enum vl_cov {
  VL_COV_EXPONENTIAL = 0, /* sigma2 exp(-h / rho)                              */
  VL_COV_MATERN15 = 1     /* sigma2 (1 + sqrt3 h / rho) exp(-sqrt3 h / rho)    */
} vl_cov;

/* Likelihood p(y_i | mu_i) (Section 2; log-concave in mu). */
typedef enum vl_lik {
  VL_LIK_BERNOULLI_LOGIT = 0, /* y in {0,1}, p = 1 / (1 + exp(-mu))             */
  VL_LIK_POISSON_LOG = 1,     /* y in {0,1,2,...}, mean exp(mu)                  */
  VL_LIK_GAMMA_LOG = 2        /* y > 0, Gamma(shape a, rate a exp(-mu)), mean exp(mu),
                               * a = opts->lik_shape (Section 5)                  */
} vl_lik;

/* Preconditioner (Section 3.1). VADU and LVA use Eqs. pcls1/logdetsplit; LRAC uses
 * Eqs. pcls2/logdetsplit2. */
typedef enum vl_precond {
  VL_PREC_VADU = 0, /* P = B^T (W + D^{-1}) B                                     */
  VL_PREC_LVA = 1,  /* P = B^T D^{-1} B                                           */
  VL_PREC_LRAC = 2  /* P = L_k L_k^T + W^{-1}, L_k pivoted Cholesky of Sigma        */
} vl_precond;

/* Arithmetic of the iterative solves. The factor build is always float64. */
typedef enum vl_precision {
  VL_FP64 = 0,        /* every Krylov vector, operator and dot in float64            */
  VL_FP32_REFINE = 1  /* float32 operator and vectors; scalars in float64; Newton
                         and simulation solves refined with float64 residuals until
                         the float64 relative residual meets cg_tol               */
} vl_precision;

typedef struct vl_opts {
  int precision;        /* vl_precision                                  default VL_FP64 */
  int precond;          /* vl_precond                                    default VL_PREC_VADU */
  int t;                /* SLQ probe vectors (Rademacher)                default 50 */
  int k;                /* LRAC rank, 1 <= k <= min(n, 1024)              default 50 */
  int s;                /* simulation vectors for predictive variances   default 100 */
  double cg_tol;        /* per-column relative residual ||r|| / ||b||    default 1e-6 */
  int cg_max_iter;      /*                                               default 1000 */
  double newton_tol;    /* max |b_new - b| <= newton_tol (1 + max |b_new|)   default 1e-9 */
  int newton_max_iter;  /*                                               default 100 */
  double nugget;        /* added to diag(Sigma); < 0 means 1e-10 sigma2  default -1 */
  uint64_t seed;        /* Philox4x64-10 key for probes and simulation   default 1 */
  double lik_shape;     /* gamma shape a > 0 (VL_LIK_GAMMA_LOG only)     default 1 */
  double newton_eta_max; /* inexact Newton: each Newton solve stops once ||rhs - A x|| <=
                            max(cg_tol ||rhs||, eta_k ||grad psi||) with the Eisenstat-Walker
                            forcing term eta_k <= newton_eta_max (capped at 0.9); the
                            iteration ends only after a solve to cg_tol. 0: every solve to
                            cg_tol                                      default 0.1 */
} vl_opts;

/* Per-call diagnostics (any pointer argument of this type may be NULL). */
typedef struct vl_stats {
  int newton_iters;
  int cg_calls;            /* PCG solves issued                                    */
  int cg_iters_max;        /* most iterations used by a column in the last solve   */
  int cg_iters_total;      /* sum of per-solve iteration counts                    */
  double cg_relres_max;    /* largest final relative residual of the last solve    */
  int refine_steps;        /* float64 refinement passes (mixed precision)          */
  double true_relres_max;  /* float64 relative residual of the refined solutions   */
  double slq_mean;         /* mean of gamma_i (the SLQ term)                       */
  double slq_stderr;       /* standard error of that mean over the probes          */
  double logdet;           /* log det(Sigma_tilde W + I) used in L^VLA             */
  double ms_total;         /* device time of the call (CUDA events)                */
  double probe_relres_max; /* vl_log_marglik: largest float64 relative residual
                              ||z - S u|| / ||z|| of the SLQ probe solves (S the
                              preconditioner's system operator); float32 solves are
                              refined until it meets cg_tol, which leaves T alone */
  int probe_refine_steps;  /* vl_log_marglik: float64 refinement passes of the probe block */
} vl_stats;

typedef struct vl_ctx vl_ctx;
typedef struct vl_factor vl_factor;
typedef struct vl_state vl_state;

/* Library version string, e.g. "vl 0.1.0 sm_103a". Never NULL. */
const char* vl_version(void);

/* Fills *o with the defaults listed in vl_opts. */
void vl_opts_default(vl_opts* o);

/* Creates a context on CUDA device `device` issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). `workspace` is a device buffer
 * of ws_bytes the library sub-allocates from for every handle made on this
 * context; if NULL, the library makes one cudaMalloc of ws_bytes here and frees it
 * in vl_ctx_destroy. Errors: VL_ERR_INVALID_ARG (out == NULL, ws_bytes < 1 MiB),
 * VL_ERR_CUDA, VL_ERR_OOM. */
vl_status vl_ctx_create(int device, void* cuda_stream, void* workspace, size_t ws_bytes,
                        vl_ctx** out);
/* Handles may be destroyed in any order: the context's stream, events and own
 * workspace are released when the context and every factor and state made on it
 * have been destroyed. A caller-provided workspace must stay allocated until then. */
void vl_ctx_destroy(vl_ctx* ctx);
/* Thread-unsafe, context-local: the message of the last failed call (or ""). */
const char* vl_last_error(const vl_ctx* ctx);
/* Blocks until the context's stream is idle. */
vl_status vl_ctx_synchronize(vl_ctx* ctx);
/* Bytes of workspace currently in use / peak use. */
vl_status vl_ctx_mem(const vl_ctx* ctx, size_t* in_use, size_t* peak);

/* Upper bound, in SM clock cycles, on each bounded device-side wait of the library's
 * kernels on this context (grid and cluster-free level barriers, the level-schedule walk);
 * 0 restores the default of 4e9 cycles (about 2 s). A wait that runs out records
 * VL_ERR_TIMEOUT and the row, makes every other wait of that launch give up at once, and
 * the call returns VL_ERR_TIMEOUT with a message; the context stays usable. Synchronises
 * the stream. VL_ERR_INVALID_ARG for cycles < 0. For tests of that path and for callers
 * that want a shorter watchdog. */
vl_status vl_ctx_set_wait_limit(vl_ctx* ctx, long long cycles);
/* Runs one bounded device-side wait on a flag that nothing sets, under the context's wait
 * limit, and returns what a library call returns when one of its waits runs out:
 * VL_ERR_TIMEOUT with its message. A check of the timeout path that every bounded wait
 * shares; the paper has no counterpart. */
vl_status vl_ctx_wait_probe(vl_ctx* ctx);

/* Launch tuning (on by default): launch parameters that change no result (blocks per SM
 * of a grid triangular solve, dependency rows in flight per lane of a block solve) are tuned
 * at first use for each (kernel class, value size, row width, size bucket): every candidate
 * runs once on the live call, timed with CUDA events, and the fastest is kept for the
 * process. enable = 0 keeps the defaults for calls on this context. */
vl_status vl_ctx_set_autotune(vl_ctx* ctx, int enable);
/* The tuner's choices so far as a JSON list (key, chosen candidate, candidate times in ms),
 * written to buf (len bytes, always NUL-terminated when len > 0); returns the bytes the
 * whole report needs, terminator included. */
size_t vl_tune_report(char* buf, size_t len);
/* Forgets every choice of the tuner: the next call of each kind tunes again (for example
 * after the device's clocks or its other load have changed). Not to be called while another
 * thread is inside a library call. */
void vl_tune_reset(void);

/* Form of the level-scheduled triangular solves with B and B^T (the two solves of the
 * VADU / LVA preconditioners, Section 3.1.1, and of Sigma_tilde = B^{-1} D B^{-T}).
 * By default each solve picks its form from n, t and the widest level; forcing one
 * serves tests (every form against the oracle) and tuning. */
typedef enum vl_solve_form {
  VL_SOLVE_AUTO = 0,    /* chosen per solve                                          */
  VL_SOLVE_SHARED = 1,  /* t = 1: one block, x in shared memory (n * sizeof <= 200 KiB);
                           block solves (t > 1) keep the automatic choice              */
  VL_SOLVE_CLUSTER = 2, /* one thread-block cluster, hardware cluster barrier per level */
  VL_SOLVE_GRID = 3,    /* cooperative grid, bounded software grid barrier per level; the
                           narrow leading and trailing levels in one block (the leading ones of
                           single-column forward solves with x in shared memory)           */
  VL_SOLVE_GRID_ALL = 4, /* cooperative grid with every level on the grid barrier         */
  VL_SOLVE_TILE = 5      /* cooperative grid of storage-row tiles, one block each; its teams
                            take the tile's rows by level and each row waits only for its
                            own dependencies (t = 1: the tile's x in shared memory). The
                            automatic choice for backward single-column solves of systems
                            above 262,144 rows                                          */
} vl_solve_form;
/* Sets the form for every later solve on this context (VL_ERR_INVALID_ARG for an
 * unknown form). A solve the forced form cannot run (VL_SOLVE_SHARED with too many
 * rows; VL_SOLVE_CLUSTER when no cluster fits the kernel, or float64 blocks wider
 * than 128 columns; VL_SOLVE_TILE when a tile of a single-column x does not fit shared
 * memory) fails with VL_ERR_INVALID_ARG. */
vl_status vl_ctx_set_solve_form(vl_ctx* ctx, int form);

/* Vecchia factor (Section 2.1): for locations `locs` (n x 2, caller order) and the
 * ordering `order` (n entries, a permutation of 0..n-1; NULL = identity; not checked here:
 * an entry outside 0..n-1 is an out-of-bounds access, the Python binding checks host arrays), finds
 * N(i) = the min(i, m) nearest earlier points under the key (d2, index) with d2 in
 * float64 and no fused multiply-add (bit-exact, ties to the lower index), the
 * forward/backward level schedules of B, and for every row the m x m covariance
 * solve A_i = Sigma_{i,N(i)} Sigma_{N(i)}^{-1}, D_i = Sigma_ii - A_i Sigma_{N(i),i}
 * with the nugget of opts on diag(Sigma). 0 <= m <= 64; n >= 1.
 * Errors: VL_ERR_INVALID_ARG, VL_ERR_NOT_SPD (row named in vl_last_error),
 * VL_ERR_OOM, VL_ERR_CUDA, VL_ERR_TIMEOUT. */
vl_status vl_build_factor(vl_ctx* ctx, const double* locs, int64_t n, const int32_t* order,
                          int cov, double sigma2, double range, int m, const vl_opts* opts,
                          vl_factor** out);

/* Recomputes A_i and D_i for new covariance parameters (the per-evaluation part of
 * Section 2.1), reusing neighbours and level schedules. */
vl_status vl_factor_refit(vl_factor* f, double sigma2, double range, const vl_opts* opts);

/* Copies the factor out in Vecchia row order (k = 0..n-1). Any pointer may be NULL.
 * N: n x m int32 (Vecchia indices, -1 padding), A: n x m float64 kriging weights
 * (B_{k,N(k)} = -A), D: n float64, lev_fwd/lev_bwd: n int32 level of each row. */
vl_status vl_factor_export(const vl_factor* f, int32_t* N, double* A, double* D,
                           int32_t* lev_fwd, int32_t* lev_bwd);
/* n, m and the number of forward / backward levels. Any pointer may be NULL. */
vl_status vl_factor_info(const vl_factor* f, int64_t* n, int* m, int* nlev_fwd, int* nlev_bwd);
void vl_factor_destroy(vl_factor* f);

/* Laplace mode (Eq. newton): b^{t+1} = (W + Sigma_tilde^{-1})^{-1}(W b^t + grad log p),
 * b^0 = 0, a step halved (at most 30 times) while it lowers
 * psi(b) = log p(y|F+b) - b^T Sigma_tilde^{-1} b / 2 by more than 1e-12 (1 + |psi|),
 * stopping when max|b^{t+1} - b^t| <= newton_tol (1 + max|b^{t+1}|). y, F (F may be NULL
 * = 0) and mode_out (may be NULL) have n entries in caller order. Every y must lie in the
 * likelihood's support (Bernoulli: 0 or 1; Poisson: a non-negative integer; gamma: > 0) and
 * y and F must be finite, else VL_ERR_INVALID_ARG naming the first offending caller index.
 * With VL_LIK_GAMMA_LOG the shape is opts->lik_shape (> 0, else VL_ERR_INVALID_ARG). A float64
 * PCG solve that stops at cg_max_iter above cg_tol is VL_ERR_NOT_CONVERGED. The state keeps b*,
 * W and the factor resident for vl_log_marglik / vl_pred_var; it references f,
 * which must outlive it. Errors: VL_ERR_NOT_CONVERGED, VL_ERR_TIMEOUT, ... */
vl_status vl_find_mode(vl_factor* f, int lik, const double* y, const double* F,
                       const vl_opts* opts, double* mode_out, vl_state** out);
void vl_state_destroy(vl_state* s);
/* Diagnostics of the Newton solve that made the state (iterations, PCG solves and
 * iterations, refinement passes, final float64 relative residual). */
vl_status vl_state_stats(const vl_state* s, vl_stats* out);

/* L^VLA (Eq. VLA_loss) at the state's mode: -log p(y|mu*) + b*^T Sigma_tilde^{-1} b* / 2
 * + log det(Sigma_tilde W + I)/2. The log-determinant is split by the preconditioner
 * (Eq. logdetsplit for VADU/LVA, Eq. logdetsplit2 for LRAC) and the last term
 * estimated by SLQ (Eq. def_SLQ) from the CG coefficients of opts->t probe solves,
 * probes z = P^{1/2} r with r Rademacher from Philox4x64-10(counter = (caller index,
 * j / 256, 0, 0), key = (seed, 0)). For LRAC the probe is z = L_k r1 + W^{-1/2} r2
 * (E z z^T = P) with r2 as above and r1 in {+-1}^k from counter (rank index, j / 256,
 * 3, 0), and log det(Sigma_tilde W + I) = log det(I_k + L_k^T W L_k) + SLQ term.
 * log p includes every constant (-log y! for Poisson). Writes the host scalars *lml
 * (and *logdet if non-NULL). */
vl_status vl_log_marglik(vl_state* s, const vl_opts* opts, double* lml, double* logdet,
                         vl_stats* stats);

/* Per-probe SLQ values gamma_i = ||P^{-1/2} z_i||^2 e1^T log(T_i) e1 of the last
 * vl_log_marglik call on this state (t doubles, host or device). */
vl_status vl_slq_gammas(const vl_state* s, double* gammas, int t);

/* Latent predictive distribution (Eq. latentpostpredictive) at np test locations
 * (np x 2): each conditions on its m nearest training points (Section 4.1, B_p = I),
 * mean_p = F_p - B_po b*, var_p = D_p + (1/s) sum_k (B_po (W + Sigma_tilde^{-1})^{-1}
 * z3_k)_p^2 with z3 = W^{1/2} z1 + B^T D^{-1/2} z2 (Algorithm simAlgo), z1, z2 standard
 * normal by Box-Muller from Philox4x64-10(counter = (caller index, j / 4, 1 or 2, 0),
 * key = (seed, 0)). Fp may be NULL (0). mean/var: np doubles (either may be NULL). */
vl_status vl_pred_var(vl_state* s, const double* test_locs, int64_t np, const double* Fp,
                      const vl_opts* opts, double* mean, double* var, vl_stats* stats);

/* Latent predictive means and variances (Eq. latentpostpredictive) at np test locations with
 * the variances from a rank-k preconditioned Lanczos factorisation (Section 4, "Predictive
 * (co-)variances using preconditioned Lanczos algorithms") instead of simulation: k steps of
 * Lanczos with full reorthogonalisation on P^{-1/2} (W + Sigma_tilde^{-1}) P^{-T/2} from
 * P^{-1/2} times the mean of the columns of B_po^T, giving
 * var_p ~ D_p + z_p^T T^{-1} z_p, z_p = Q^T P^{-1/2} B_po^T e_p (fewer than k steps when the
 * Krylov space closes). precond_l selects the Lanczos preconditioner: 1 = P_L1 =
 * B^T (W + D^{-1}) B (the only one available; others: VL_ERR_INVALID_ARG). Float64. The
 * estimate is biased low for small k and exact at k = n. mean/var: np doubles (either may be
 * NULL); stats->cg_iters_max receives the number of Lanczos steps taken. */
vl_status vl_pred_var_lanczos(vl_state* s, const double* test_locs, int64_t np, const double* Fp,
                              int k, int precond_l, double* mean, double* var, vl_stats* stats);

/* Kernel timing. While enabled (enable >= 1), every launch of the library's hot kernels is
 * bracketed by a pair of CUDA events on the context's stream, grouped by kernel
 * class and block width: "sptrsv_fwd", "sptrsv_bwd", "spmv_B", "spmv_Bt",
 * "pcg_update", "coldot", "factor", "knn", and for LRAC "woodbury" (one
 * preconditioner apply), "lrac_gram" and "lrac_kxk" (at width k: C = I + L^T W L,
 * its Cholesky factor and inverse) and "pivoted_cholesky" (at width k). Costs two
 * event records per launch group. */
vl_status vl_profile_enable(vl_ctx* ctx, int enable);
/* With enable >= 2 every triangular solve also records block 0's SM clock at each
 * level boundary; this returns the last such trace of class `cls` ("sptrsv_fwd" /
 * "sptrsv_bwd") at block width t: *len = levels + 1 clock values (cycles), and the
 * head / tail level cut used (levels [0, l_head) and [l_tail, nlev) ran in block 0
 * alone). Costs a stream synchronisation per solve. */
vl_status vl_profile_trace(vl_ctx* ctx, const char* cls, int t, long long* out, int cap, int* len,
                           int* l_head, int* l_tail);
/* Device time (ms, summed) and launch count of class `cls` at block width t
 * (t = 0: all widths) since the last reset; reset != 0 clears every class.
 * cls = "all" gives the number of kernels launched on the context (counted
 * whether or not profiling is enabled) and zero time. Synchronises the stream.
 * Unknown class: zero time and count. */
vl_status vl_profile_read(vl_ctx* ctx, const char* cls, int t, double* ms, int64_t* launches, int reset);

/* ------------------------------------------------------------------------------
 * Building blocks, exposed for verification and for callers composing their own
 * solvers. Vectors are in caller order, n x t row-major float64.
 * ---------------------------------------------------------------------------- */

/* The m nearest earlier neighbours of every point of `locs` (n x 2) taken in the
 * given row order (Section 2.1; key (d2, index), bit-exact). N_out: n x m int32. */
vl_status vl_knn_prev(vl_ctx* ctx, const double* locs, int64_t n, int m, int32_t* N_out);
/* The min(m, n) nearest training points of each test point (Section 4.1), same key.
 * N_out: np x m int32 (training row indices, -1 padding). */
vl_status vl_knn_cross(vl_ctx* ctx, const double* train, int64_t n, const double* test,
                       int64_t np, int m, int32_t* N_out);

typedef enum vl_op {
  VL_OP_A = 0,        /* (W + B^T D^{-1} B) X                                     */
  VL_OP_PINV = 1,     /* P^{-1} X for the state's preconditioner (opts->precond)    */
  VL_OP_B = 2,        /* B X                                                       */
  VL_OP_BT = 3,       /* B^T X                                                     */
  VL_OP_BINV = 4,     /* B^{-1} X  (level-scheduled forward solve)                  */
  VL_OP_BTINV = 5,    /* B^{-T} X  (level-scheduled backward solve)                 */
  VL_OP_SIGMA = 6,    /* Sigma_tilde X = B^{-1} D B^{-T} X                          */
  VL_OP_A2 = 7        /* (Sigma_tilde + W^{-1}) X  (the form-2 operator, Eq. pcls2)  */
} vl_op;

/* Y = op(X) with the state's W, in the precision of opts (float64 in/out). */
vl_status vl_apply(vl_state* s, int op, const double* X, int t, const vl_opts* opts, double* Y);

/* Y = (W + B^T D^{-1} B) X in float64, like vl_apply(VL_OP_A), but without touching
 * the context workspace or allocating device memory, for callers that cannot
 * allocate when they call: its intermediates live in a fixed 64 MiB array built
 * into the library (resident on every device that loads it), so it requires
 * 3 * n * ld * 8 + n * 8 <= 64 MiB with ld = 1 for t = 1, else 8 * ceil(t / 8);
 * larger requests fail with VL_ERR_INVALID_ARG and say so. X and Y must be device
 * pointers (n x t, caller order). The first call on a device looks up the array's
 * address, so make it before any stream capture. Calls share the array: calls that
 * overlap on the GPU race. The paper has no counterpart; this is a deployment aid. */
vl_status vl_apply_A_noalloc(vl_state* s, const double* X, int t, double* Y);

/* Solves the preconditioner's system by PCG with T extraction (the appendix
 * algorithm, u_0 = 0, per-column stop ||r|| <= cg_tol ||b||), in the precision and
 * preconditioner of opts: (W + Sigma_tilde^{-1}) U = RHS for VADU and LVA (Eq. pcls1),
 * (Sigma_tilde + W^{-1}) U = RHS for LRAC (Eq. pcls2).
 * T_diag/T_off: t x lmax row-major (may be NULL), iters: t ints (may be NULL),
 * relres: t doubles (may be NULL). */
vl_status vl_pcg_solve(vl_state* s, const double* RHS, int t, const vl_opts* opts, double* U,
                       int lmax, double* T_diag, double* T_off, int* iters, double* relres);

/* Gradient of L^VLA with respect to (sigma2, range) at the state's mode (appendix
 * "Gradients of Vecchia-Laplace approximations"): grad[0] = dL/dsigma2, grad[1] = dL/drange
 * (host doubles), with every log-determinant derivative by stochastic trace estimation
 * (Eq. grad_STE) on the opts->t probes of vl_log_marglik (same seed, same z = P^{1/2} r) and
 * the control variate r(z) = z^T P^{-1} dP P^{-1} z with weight c = Cov(h, r) / Var(r)
 * (Section 3; c = 0 when r does not vary over the probes), and the implicit dependence through
 * the mode by one more solve with W + Sigma_tilde^{-1}. The nugget is taken to scale with sigma2.
 * dF (n doubles, caller order, host or device; may be NULL) receives dL/dF =
 * -grad log p(y | mu*) + g - W (W + Sigma_tilde^{-1})^{-1} g with g = 1/2 dlogdet/dmu* by the
 * same estimator. Supported: VL_FP64 with VL_PREC_VADU, Bernoulli or Poisson likelihood
 * (VL_ERR_INVALID_ARG otherwise). */
vl_status vl_lml_grad(vl_state* s, const vl_opts* opts, double* grad, double* dF, vl_stats* stats);

/* ------------------------------------------------------------------------------
 * Batches: independent problems (the same method, Sections 2-3, applied to each) merged into
 * one block-diagonal system. The rows of the problems are concatenated and the level sets of
 * their triangular factors merged level by level, so one launch of every kernel serves all
 * problems and a triangular solve takes as many levels as the deepest problem. Reductions
 * are per problem and the Newton and PCG scalars per (problem, column): each problem follows
 * its own Newton iteration and its own PCG stopping rule, with the probes and tolerances it
 * would have alone (results equal the problems solved one by one, up to rounding).
 * Vectors of a batch are the problems' vectors concatenated in problem order, each in its
 * problem's caller order.
 * ---------------------------------------------------------------------------- */
typedef struct vl_batch vl_batch;
/* Merges nprob factors made by vl_build_factor on ctx (they must outlive the batch; any m,
 * covariance and size). Copies their neighbour tables, weights and level schedules.
 * Errors: VL_ERR_INVALID_ARG, VL_ERR_OOM. */
vl_status vl_batch_create(vl_ctx* ctx, int nprob, vl_factor* const* factors, vl_batch** out);
/* Copies the members' factor values again after vl_factor_refit of any of them. */
vl_status vl_batch_refresh(vl_batch* b);
/* Total rows and the levels of the merged forward / backward solves (pointers may be NULL). */
vl_status vl_batch_info(const vl_batch* b, int64_t* n_total, int* nlev_fwd, int* nlev_bwd);
/* Laplace modes of every problem (Eq. newton, as vl_find_mode): lik[k] is problem k's
 * likelihood (a gamma problem takes opts->lik_shape); y, F (F may be NULL = 0) and mode_out
 * (may be NULL) hold sum n_k values; stats (NULL or nprob entries) receives each problem's
 * Newton statistics. VADU or LVA preconditioner. The batch keeps the modes for
 * vl_batch_log_marglik. VL_ERR_NOT_CONVERGED if any problem stops at newton_max_iter. */
vl_status vl_batch_find_mode(vl_batch* b, const int* lik, const double* y, const double* F,
                             const vl_opts* opts, double* mode_out, vl_stats* stats);
/* L^VLA of every problem at its mode (as vl_log_marglik, each problem with its own opts->t
 * probes): lml[k] (host, nprob), logdet (NULL or nprob), stats (NULL or nprob). */
vl_status vl_batch_log_marglik(vl_batch* b, const vl_opts* opts, double* lml, double* logdet,
                               vl_stats* stats);
/* Predictive means and simulated variances of every problem (as vl_pred_var: Eq.
 * latentpostpredictive, Algorithm simAlgo with opts->s vectors drawn by each problem's own
 * caller indices): np[k] test points of problem k, their locations (sum np x 2) and offsets Fp
 * (sum np, may be NULL) concatenated in problem order; mean and var (sum np each, host or
 * device, either may be NULL). Each test point conditions on the m_k nearest training points of
 * its own problem. Call after vl_batch_find_mode. */
vl_status vl_batch_pred_var(vl_batch* b, const int64_t* np, const double* test_locs, const double* Fp,
                            const vl_opts* opts, double* mean, double* var);
/* SLQ values of the last vl_batch_log_marglik: nprob x t host doubles, problem-major. */
vl_status vl_batch_gammas(const vl_batch* b, double* gammas, int t);
void vl_batch_destroy(vl_batch* b);

/* The rank-k pivoted Cholesky factor L_k of Sigma used by the LRAC preconditioner
 * (Section 3.1.2; Harbrecht, Peters & Schneider 2012): residual diagonal d = diag Sigma
 * (nugget included), k steps of pivot p = argmax d (ties to the lowest Vecchia index),
 * L[:, j] = (Sigma[:, p] - L[:, :j] L[p, :j]^T) / sqrt(d_p), d -= L[:, j]^2, d_p = 0, in
 * float64. Built on first use and kept with the factor until vl_factor_refit.
 * piv: k int32 Vecchia indices of the pivots (may be NULL); L: n x k float64,
 * caller order, row-major (may be NULL). Errors: VL_ERR_INVALID_ARG (k outside
 * [1, min(n, 1024)]), VL_ERR_NOT_SPD (d_p <= 0 before step k: Sigma has numerical
 * rank < k), VL_ERR_OOM. */
vl_status vl_lrac_export(vl_factor* f, int k, int32_t* piv, double* L);

#ifdef __cplusplus
}
#endif
#endif /* VL_H_ */
