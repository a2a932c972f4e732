/*
 * libfde -- GB300 (sm_103a) solver for the per-time-step linear system of the
 * CN-WSGD discretisation of the two-dimensional two-sided space-fractional
 * diffusion equation, after Moghaderi, Dehghan, Donatelli, Mazza,
 * "Spectral analysis and multigrid preconditioners for two-dimensional
 * space-fractional diffusion equations" (arXiv:1706.06844).
 *
 * At each time step t^(m) the scheme (Sec. 2, Eq. CNWSGD) leaves
 *     M u^(m) = b^(m),                                           (Eq. 2)
 *     M = c I + D+ (I (x) A_alpha) + D- (I (x) A_alpha^T)
 *           + sigma [E+ (A_beta (x) I) + E- (A_beta^T (x) I)],   (Eq. M, AxAy)
 *     b = (c I - A_x^(m-1) - sigma A_y^(m-1)) u^(m-1) + 2 hx^alpha v^(m-1/2),
 * with A_gamma = -[w_{i-j+1}] (Eq. AN), w the WSGD weights (Eq. w),
 * c = 1/r = 2 hx^alpha / dt and sigma = s/r = hx^alpha / hy^beta.  The system
 * is solved by restarted flexible GMRES (Sec. 5) preconditioned by one
 * multigrid V-cycle (Sec. 4: damped Jacobi, bilinear interpolation, Galerkin
 * or rediscretised coarse operators) or by the band preconditioner P_2 with a
 * Galerkin V-cycle (Sec. 4.3); multigrid can also run as the solver itself.
 *
 * Conventions shared by every call:
 *  - Grid functions are row-major n2 x n1 arrays U[j][i] of doubles, x index i
 *    fastest (the lexicographic ordering of Sec. 2), no padding: element
 *    (i, j) is at U[j * n1 + i].
 *  - Unless a name ends in _host, every pointer argument is DEVICE memory owned
 *    by the caller; the library reads/writes it on the handle's stream and keeps
 *    no reference after the call returns.  The library owns its workspace
 *    (Krylov basis, multigrid hierarchy, weights), allocated in fde_create and
 *    freed in fde_destroy.
 *  - Every call returns an int status: FDE_OK (0) or one of the FDE_ERR_*
 *    codes; fde_last_error gives a message.  Argument errors are detected on
 *    the host before any launch.  Calls that run a solve (fde_solve, fde_step,
 *    fde_step_host) synchronise the stream before returning; the others only
 *    enqueue work (their outputs are valid after a stream synchronisation).
 *  - A handle is not thread-safe; separate handles are independent.
 */
#ifndef FDE_H
#define FDE_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FDE_OK                 0
#define FDE_ERR_ARG            1  /* invalid argument (bad size, order, null pointer ...) */
#define FDE_ERR_NOT_CONVERGED  2  /* maxit reached; the output holds the last iterate */
#define FDE_ERR_NONFINITE      3  /* NaN/Inf met in a residual norm */
#define FDE_ERR_CUDA           4  /* a CUDA runtime call failed */
#define FDE_ERR_TIMEOUT        5  /* a capped device-side wait gave up */
#define FDE_ERR_UNSUPPORTED    6  /* valid request this build does not implement */

/* preconditioner (Sec. 4) */
#define FDE_PRECOND_NONE       0  /* plain GMRES */
#define FDE_PRECOND_MG_SG      1  /* V-cycle, structured Galerkin coarse operators, R = P^T */
#define FDE_PRECOND_MG_REDISC  2  /* V-cycle, rediscretised coarse operators, R = P^T / 4 (P_MGM, Sec. 4.2) */
#define FDE_PRECOND_P2         3  /* band preconditioner P_2 (Sec. 4.3): Laplacian (alpha = beta = 2)
                                     five-point operator with the problem's coefficients, one
                                     Galerkin V-cycle (nine-point coarse stencils, R = P^T) */
#define FDE_PRECOND_MG_EXACT   4  /* V-cycle with the exact Galerkin coarse operators
                                     A_{l+1} = P^T A_l P as dense matrices formed on the device
                                     (Sec. 4, TGM step 3; the paper's tilde-P_MGM, Sec. 5.1):
                                     a validation mode for small grids, n1 n2 <= 4096, FP64 only */

/* arithmetic of the preconditioner (the outer Krylov method is FP64-accurate: see FDE_OUTER_*) */
#define FDE_PREC_FP64          0  /* V-cycle in FP64 ("plain FP64" solver) */
#define FDE_PREC_FP32          1  /* V-cycle vectors and Toeplitz products in FP32 */
#define FDE_PREC_BF16          2  /* FP32 vectors, Toeplitz products on tcgen05 in BF16 with FP32 accumulation */
#define FDE_PREC_FP16          3  /* as BF16 with FP16 operands */
#define FDE_PREC_BF16X3        4  /* operands split into BF16 hi + lo, three tcgen05 products per block
                                     accumulated in FP32 (~16-bit operands) */

/* how the preconditioner's dense Toeplitz products are evaluated */
#define FDE_PATH_AUTO          0  /* tensor-core GEMM for BF16/FP16/BF16X3 on levels with n >= 1536, else FFT
                                     above the direct-sum cut-off (n >= 127), else direct */
#define FDE_PATH_GEMM          1  /* tcgen05 GEMM (BF16/FP16/BF16X3 only) */
#define FDE_PATH_FFT           2  /* circulant-embedding FFT */
#define FDE_PATH_DIRECT        3  /* direct summation */
#define FDE_PATH_TUNE          4  /* on the first coefficient set-up every level times its
                                     candidate paths on the device -- tensor cores (BF16/FP16/
                                     BF16X3, n >= 127), FFT, direct summation (n <= 1023) -- and
                                     keeps the fastest (a later path in that order only when
                                     faster by more than 3 %) */

/* arithmetic of the FP64-accurate outer apply (Krylov matvec, true residual, rhs) */
#define FDE_OUTER_FP64         0  /* FFT in FP64; FGMRES vectors and Gram-Schmidt in FP64 */
#define FDE_OUTER_DF32         1  /* FFT in double-float (pairs of FP32), ~48-bit significand;
                                     with restart <= 32 the single-problem FGMRES also keeps its
                                     basis vectors in double-float and runs Gram-Schmidt on the
                                     FP32 pipes (x, b and the true residual stay FP64; the
                                     Hessenberg matrix, rotations and least squares are FP64) */

/* coefficient time levels */
#define FDE_COEF_NEW           0  /* d+-, e+- at t^(m): the system matrix M^(m) */
#define FDE_COEF_OLD           1  /* d+-, e+- at t^(m-1): the right-hand side b^(m) */

typedef struct fde_params {
  double alpha, beta;      /* fractional orders in (1, 2) (problem (1), Sec. 2) */
  int    qx, qy;           /* WSGD shift q, with p = 1: 0 is Eq. (w); -1 is the (1,-1) member of
                              the same weighted-and-shifted family */
  double a1, b1, a2, b2;   /* domain (a1, b1) x (a2, b2) */
  int    n1, n2;           /* interior points; hx = (b1-a1)/(n1+1), hy = (b2-a2)/(n2+1) (Sec. 2) */
  double dt;               /* time step */
  double rtol;             /* stop when ||b - M x||_2 <= rtol ||b||_2 (true residual) */
  int    restart;          /* FGMRES restart length m (1 .. 64) */
  int    maxit;            /* cap on total inner iterations per solve */
  int    precond;          /* FDE_PRECOND_* */
  int    nu_pre, nu_post;  /* Jacobi sweeps before / after the coarse correction (0 .. 4) */
  double omega;            /* Jacobi damping (Lemma lemsmo: 0 < omega < 2 a_0/||F||_inf) */
  int    coarsest_n;       /* coarsen while n > coarsest_n (the paper fixes an 8 x 8 grid) */
  int    precision;        /* FDE_PREC_* */
  int    toeplitz_path;    /* FDE_PATH_* */
  int    outer;            /* FDE_OUTER_* */
  int    cycles;           /* V-cycles per preconditioner application (0 or 1: one; at most 4);
                              cycle k + 1 corrects the residual of cycle k (Sec. 5.1 tries two
                              for P_2).  When n1 or n2 <= coarsest_n the hierarchy has one
                              level, the cycle is the exact coarsest-grid solve, and the
                              Toeplitz preconditioners run it once */
  int    relax;            /* 1: relaxed Krylov matvec -- once the FGMRES residual estimate is
                              within FDE_RELAX_FACTOR of rtol ||b||, M z is evaluated in FP32
                              (inexact Krylov: matvec errors eta_j with
                              eta_j ||r_{j-1}|| <= rtol ||b|| / m keep the final residual within
                              rtol; an FP32 FFT apply has eta ~ 1e-6 relative to ||M|| ||z||,
                              so the switch at 1e4 x the target leaves a margin of ~10 at
                              m = 13); the right-hand side and every true residual stay
                              FP64-accurate, so the stopping test is unchanged.  0 (default):
                              every matvec FP64-accurate, as in the paper's GMRES. */
  int    solver;           /* FDE_SOLVER_FGMRES (default) or FDE_SOLVER_MG: multigrid as the
                              solver itself, x <- x + V(b - M x) until the true residual meets
                              rtol (Sec. 1 and Sec. 4.3: the multigrid method can run without a
                              Krylov wrapper); restart is ignored, maxit caps the cycles */
  int    warm;             /* 1: fde_step starts the solve from u_prev instead of zero (the
                              paper starts from zero, Sec. 5) */
} fde_params;

#define FDE_SOLVER_FGMRES 0
#define FDE_SOLVER_MG     1

#define FDE_RELAX_FACTOR 1.0e4

typedef struct fde_stats {
  int    iterations;       /* inner FGMRES steps (= preconditioner applications) */
  int    restarts;         /* restart cycles begun */
  int    converged;        /* 1 if the true residual met rtol */
  double rel_residual;     /* ||b - M x||_2 / ||b||_2 at exit, true residual in FP64 */
  int    relaxed;          /* Krylov matvecs evaluated in FP32 (fde_params.relax) */
} fde_stats;

typedef struct fde_handle fde_handle;

/* Fill *p with defaults: alpha = beta = 1.5, q = 0, unit square, n = 63,
 * dt = h, rtol 1e-8, FGMRES(30), maxit 1000, MG_SG, nu = (1, 1), omega 0.7,
 * coarsest 8, FP64, AUTO path, FP64 outer apply, one V-cycle. */
void fde_default_params(fde_params* p);

/* Create a solver for one grid (Sec. 2).  Checks the parameters, allocates
 * the workspace and generates the WSGD weights w_0..w_n (Eq. gk, Eq. w) on
 * the device in FP64.  `stream` is a cudaStream_t (NULL = legacy default).
 * Coefficients must be set (fde_set_coefficients) before any apply or solve.
 * Levels coarsen n -> (n - n mod 2)/2 (Sec. 4.1's K matrix: coarse j on fine
 * 2j for odd n, 2j - 1 for even n) down to <= coarsest_n; the structured-
 * Galerkin hierarchy (MG_SG) needs every level size odd, the others take
 * either parity.
 * On error *out is NULL and the status says why. */
int fde_create(const fde_params* p, void* stream, fde_handle** out);

/* Free the workspace.  NULL is a no-op. */
void fde_destroy(fde_handle* h);

/* Last error message of `h`, or of the last failed fde_create when h is NULL. */
const char* fde_last_error(const fde_handle* h);

/* Set the diffusion coefficients d+, d-, e+, e- (Sec. 2: the diagonals of
 * D+-, E+-) sampled on the grid, each an n2 x n1 device array.  `which` is
 * FDE_COEF_NEW (t^(m): builds M and the multigrid hierarchy -- coarse
 * coefficients by injection, level diagonals, coarse Toeplitz factors -- on
 * the device) or FDE_COEF_OLD (t^(m-1): used only by fde_rhs / fde_step).
 * The arrays are copied; the caller may free them afterwards. */
int fde_set_coefficients(fde_handle* h, int which, const double* dp, const double* dm,
                         const double* ep, const double* em);

/* b = (c I - A_x^(m-1) - sigma A_y^(m-1)) u_prev + 2 hx^alpha v_half  (Eq. M,
 * second line), with the FDE_COEF_OLD coefficients.  FP64-accurate. */
int fde_rhs(fde_handle* h, const double* u_prev, const double* v_half, double* b);

/* y = M x (Eq. M) with the FDE_COEF_NEW coefficients; FP64-accurate (the
 * outer apply chosen by params.outer).  x and y must not alias. */
int fde_apply(fde_handle* h, const double* x, double* y);

/* z = B r: one application of the preconditioner (one V-cycle from a zero
 * initial guess, Sec. 4 and 4.2), in the configured precision.  With
 * FDE_PRECOND_NONE, z = r. */
int fde_vcycle(fde_handle* h, const double* r, double* z);

/* y = K_l x for multigrid level l (0 = finest), the level operator the
 * V-cycle uses, in the configured precision.  x, y are n2_l x n1_l arrays. */
int fde_level_apply(fde_handle* h, int level, const double* x, double* y);

/* Number of multigrid levels and their sizes (arrays of length >= levels;
 * either may be NULL). */
int fde_levels(const fde_handle* h, int* levels, int* n1s, int* n2s);
/* Product path (FDE_PATH_GEMM / FFT / DIRECT) a Toeplitz multigrid level
 * uses; -1 for the coarsest level (dense inverse), P_2 stencil levels, a
 * handle without multigrid or an invalid level. */
int fde_level_path(const fde_handle* h, int level);

/* Copy the device-generated WSGD weights w_0..w_{count-1} of axis 0 (x,
 * alpha) or 1 (y, beta) to host memory. */
int fde_weights(const fde_handle* h, int axis, double* w_host, int count);

/* Solve M x = b (Eq. 2) from x = 0: by FGMRES(restart), right
 * preconditioned (Sec. 5), or with params.solver = FDE_SOLVER_MG by the
 * stationary multigrid iteration.  Writes x even when not converged
 * (FDE_ERR_NOT_CONVERGED).  FDE_ERR_NONFINITE: NaN/Inf in a residual norm.
 * FDE_ERR_TIMEOUT: a capped wait of a tensor-core kernel gave up during the
 * solve (x is written; the flag is cleared, so the handle stays usable).
 * `st` may be NULL.  Synchronises the stream. */
int fde_solve(fde_handle* h, const double* b, double* x, fde_stats* st);

/* One CN-WSGD time step (Eq. CNWSGD): b from u_prev, v_half and the OLD
 * coefficients, then the solve of fde_solve (started from u_prev instead of
 * zero when params.warm = 1).  u_next must not alias u_prev.  Increments the
 * step counter. */
int fde_step(fde_handle* h, const double* u_prev, const double* v_half, double* u_next,
             fde_stats* st);

/* fde_step with HOST arrays: copies u_prev and v_half host->device, runs the
 * step and copies u_next device->host (pageable or page-locked host memory).
 * With page-locked arrays the copies overlap the computation on a second
 * stream of the handle (created on the first call): v_half uploads while the
 * right-hand side's operator apply of u_prev runs, and every FGMRES cycle's
 * solution is copied to u_next while its true residual is checked (the last
 * copy is the result).  All copies are complete when the call returns. */
int fde_step_host(fde_handle* h, const double* u_prev_host, const double* v_half_host,
                  double* u_next_host, fde_stats* st);

/* Checkpoint: the step counter m and the last solution written by fde_step
 * (copied to u_out, device memory, may be NULL). */
int fde_get_state(const fde_handle* h, int* m, double* u_out);
/* Restore the step counter (the caller keeps u^(m) and passes it to fde_step). */
int fde_set_state(fde_handle* h, int m);

/* Failure-path self-test of the tensor-core kernels (no paper passage: a
 * property of this implementation).  Enqueues on the handle's stream one
 * run of those kernels' bounded mbarrier wait, in a one-warp kernel, on a
 * barrier that is completed (complete = 1) or that nothing completes
 * (complete = 0: the wait gives up after 20 ms and raises the device error
 * flag of the handle's first tensor-core level, as a products kernel whose
 * wait ran out would).  Nothing faults or hangs.  The flag is read by the
 * next fde_solve / fde_step, which then returns FDE_ERR_TIMEOUT (once; the
 * flag is cleared when read) after writing its result as usual.  Returns
 * FDE_OK when enqueued, FDE_ERR_ARG for a NULL handle or complete not 0/1,
 * FDE_ERR_UNSUPPORTED if the handle has no tensor-core level, FDE_ERR_CUDA
 * on a launch error.  Does not synchronise. */
int fde_wait_selftest(fde_handle* h, int complete);

/* Self-test of the integer-only number conversions the kernels use instead
 * of FP64 instructions (no paper passage: GB300 runs FP64 arithmetic and
 * conversions at 1/64 of the FP32 rate).  On the current device, n seeded
 * inputs (random bit patterns of every exponent, values near the FP32 range
 * and its edges, rounding ties, zeros, subnormals, infinities, NaN) compare
 * double -> float (round to nearest even) and float -> double with the CUDA
 * conversions bit for bit (NaN as NaN), and the double -> double-float split
 * with its bounds |hi + lo - x| <= 2^-47 |x| for 2^-73 <= |x| <= 2^100 and
 * <= 2^-97 below.
 * *mismatches (host) receives the number of failures.  Returns FDE_OK,
 * FDE_ERR_ARG for n < 1 or a NULL pointer, FDE_ERR_CUDA on a CUDA error.
 * Synchronises the device. */
int fde_conversion_selftest(long long n, long long* mismatches);

/* Kernel-level timing with CUDA events on the handle's stream (off by
 * default).  Kernel classes: FDE_KCLASS_*.  fde_profile_query returns the
 * number of launches and their summed event time since the last reset. */
#define FDE_KCLASS_OUTER_APPLY  0  /* FP64-accurate Toeplitz apply, whole apply (both FFT passes
                                      and the transposes of the column pass) */
#define FDE_KCLASS_LEVEL_APPLY  1  /* preconditioner Toeplitz products (incl. operand packing) */
#define FDE_KCLASS_KRYLOV       2  /* Arnoldi / update / norm kernels */
#define FDE_KCLASS_MG_OTHER     3  /* smoother, transfers, coarse solve */
#define FDE_KCLASS_OUTER_FP32   4  /* relaxed (FP32) Krylov matvecs, whole apply */
#define FDE_KCLASS_TC_GEMM      5  /* each tcgen05 products launch (one direction) on its own;
                                      these launches are also counted in LEVEL_APPLY */
#define FDE_KCLASS_COUNT        6
int fde_profile_enable(fde_handle* h, int on);
int fde_profile_query(fde_handle* h, int kclass, long long* launches, double* ms);
/* Total kernels this handle has launched. */
long long fde_launch_count(const fde_handle* h);

/* Batch of independent problems (Sec. 2's scheme on each, sizes, orders and
 * coefficients may all differ), stepped together: by the grouped engine (see
 * fde_batch_engine) or by up to 16 host worker threads (the environment
 * variable FDE_BATCH_WORKERS, 1..256, read at creation, overrides the cap),
 * each with its own CUDA stream, running disjoint subsets of the problems
 * (largest first).  params[0..count) are copied; problem i gets a
 * handle of its own (fde_batch_handle) on which the caller sets coefficients
 * or state as for a single problem.  Work of fde_batch_step starts after the
 * work already enqueued on `stream` and `stream` waits for all of it before
 * anything enqueued later; the call returns when every solve has finished.
 * The batch owns its handles; do not destroy them separately.  Errors:
 * FDE_ERR_ARG (null params, count <= 0), or the first failing problem's
 * fde_create status; message via fde_last_error(NULL). */
typedef struct fde_batch fde_batch;
int fde_batch_create(const fde_params* params, int count, void* stream, fde_batch** out);
void fde_batch_destroy(fde_batch* b);
int fde_batch_size(const fde_batch* b);
/* Handle of problem i (NULL when i is out of range). */
fde_handle* fde_batch_handle(fde_batch* b, int i);
/* One CN step of every problem i: fde_step(handle i, u_prev[i], v_half[i],
 * u_next[i], st + i).  The three arrays hold `count` DEVICE pointers (host
 * arrays of device pointers); st may be NULL or hold `count` entries.  Every
 * problem is stepped even when another fails; returns FDE_OK or the status of
 * the lowest-numbered failing problem (fde_last_error(NULL) names it, and
 * fde_batch_status gives each problem's own status). */
int fde_batch_step(fde_batch* b, const double* const* u_prev, const double* const* v_half,
                   double* const* u_next, fde_stats* st);
int fde_batch_status(const fde_batch* b, int i);
/* Which engine stepped the batch: 0 none yet, 1 grouped (every stage of all
 * problems' solves -- Toeplitz passes, transposes, smoothing, transfers, the
 * V-cycle tail, matvecs, Gram-Schmidt passes, Givens updates -- one launch for
 * the whole batch, FGMRES iterations in lockstep with per-problem gates on the
 * device, one restart cycle of the batch replayed from a CUDA graph), 2 worker
 * threads.  The grouped engine is used when every problem runs the FP32
 * V-cycle (MG_SG or MG_REDISC, FFT or direct-sum products above the
 * one-launch tail, one cycle per application), the double-float outer apply,
 * FGMRES with one restart length <= 32 and no warm start, unless the
 * environment variable FDE_BATCH_ENGINE=threads (read at the first step) asks
 * for the worker threads; fde_batch_engine_note says why an engine was chosen. */
int fde_batch_engine(const fde_batch* b);
const char* fde_batch_engine_note(const fde_batch* b);
/* Kernels launched for the batch so far (both engines, graph nodes counted). */
long long fde_batch_launch_count(const fde_batch* b);

/* y = M x (Eq. M) with the given coefficients (device arrays d+, d-, e+, e-,
 * n2 x n1, as for fde_set_coefficients) in FP64, WITHOUT a handle and WITHOUT
 * allocating device memory: for callers that cannot allocate GPU memory (the
 * device heap is owned by another runtime's fixed pool or allocator, or the
 * process must not grow its device footprint), and who therefore cannot call
 * fde_create.  The paper has no counterpart; it is a deployment convenience.
 * Only alpha, beta, qx, qy, a1, b1, a2, b2, n1, n2 and dt of *p are read.
 * Grids larger than 2048 points on either axis are rejected (FDE_ERR_ARG):
 * the working data (weights, spectra, twiddles, about 450 KB) lives in one
 * fixed device array that every GPU loading the library holds until exit.
 * The first call on a device looks that array up (cudaGetSymbolAddress) with
 * the device current and keeps the address; make that first call before any
 * stream capture, and do not reset the device (cudaDeviceReset) between calls:
 * a kept address would then be stale.  y must not overlap x or a coefficient
 * array (FDE_ERR_ARG).  Each
 * call rewrites the array before using it; calls that overlap on the GPU
 * (other streams or host threads) race on it and must be serialised by the
 * caller.  Work is enqueued on `stream`; errors via fde_last_error(NULL). */
int fde_apply_noalloc(const fde_params* p, const double* dp, const double* dm,
                      const double* ep, const double* em, const double* x, double* y,
                      void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FDE_H */
