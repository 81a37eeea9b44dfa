/*
 * curldiv.h — C ABI of the GB300 (sm_103a) solver library for the isogeometric
 * curl-div problem
 *
 *     alpha (curl u, curl v) + beta (div u, div v) = (f, v)   for all v in V_h
 *
 * (Section 1, eq:curl-div), discretised with tensor-product B-splines of degree p
 * on n uniform intervals per direction of the unit square (d = 2) or cube
 * (d = 3), homogeneous Dirichlet conditions imposed strongly (Section 3.1,
 * eq:tensor2D).  The Galerkin matrix is eq:matr_Amu (d = 2) / eq:matr_Amu3D
 * (d = 3); the linear system solved is eq:system, A w = b.
 *
 * Vector layout (every entry point, host or device): FP64 (or FP32 where the name
 * says so), C order [nrhs][d][m]...[m] with m = n + p - 2, i.e. component-major
 * (w = [u^1; ...; u^d], Section 4, eq:eq_1) and, inside a component, the
 * Kronecker order of the tensor index with x_1 slowest and x_d fastest.  One
 * right-hand side has d * m^d entries (cd_dofs).
 *
 * Parameters: each entry point that takes `alphas` / `betas` reads nrhs host
 * doubles (one (alpha, beta) pair per right-hand side, so one batched call can
 * mix parameters); NULL means "the handle's alpha / beta for every RHS".  Every
 * alpha and beta must be finite and > 0 (A is then SPD, Section 5, Thm 5.2/5.6).
 *
 * Ownership: the caller owns every vector it passes (device pointers unless the
 * name ends in _host).  The library owns all of its device state (1D bands, the
 * multigrid hierarchy, eigenbases, workspace, captured graphs); cd_destroy frees it.
 * All device work is ordered on the stream given to cd_create.
 *
 * Errors: every entry point returns a cd_status and never throws or aborts
 * across the ABI.  CD_EINVAL: bad dimension (d not 2 or 3, p < 1, n < 1,
 * m < 2, d m^d >= 2^31), non-finite or non-positive parameter, NULL pointer, nrhs < 1 or above
 * the handle's batch capacity.  CD_ECUDA: a CUDA call failed (the text is
 * available from cd_last_error).  CD_NOT_CONVERGED: maxit reached; x holds the
 * last iterate and cd_result its residual.  CD_BREAKDOWN: a Krylov denominator
 * was <= 0 or not finite (for example a NaN right-hand side).
 */
#ifndef CURLDIV_H
#define CURLDIV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CD_API __attribute__((visibility("default")))

typedef struct cd_solver_s* cd_solver;

typedef enum {
  CD_OK = 0,
  CD_EINVAL = 1,
  CD_ENOMEM = 2,
  CD_ECUDA = 3,
  CD_NOT_CONVERGED = 4,
  CD_BREAKDOWN = 5,
  CD_TIMEOUT = 6,
  CD_CANCELLED = 7
} cd_status;

/* Arithmetic of the solve.  Both modes run an outer loop that measures the true
 * residual b - A x in FP64 and updates x in FP64; they differ in the inner solve.
 * CD_PREC_FP64: every kernel in FP64 (operator, Krylov vectors, preconditioner); the
 *   outer loop only restarts the Krylov solve when its recursive residual has
 *   drifted from the true one.
 * CD_PREC_FP32_IR: iterative refinement.  A right-hand side whose parameter ratio
 *   max(alpha, beta) / min(alpha, beta) is below `mixed_switch_ratio` gets an inner
 *   preconditioned Krylov solve whose operator, vectors and preconditioner are FP32
 *   (inner products in FP64).  Above the ratio, or after an FP32 refinement step
 *   that reduced the residual less than tenfold, its inner solve is FP64 throughout:
 *   in FP32 the contribution of the small parameter to A w cancels below rounding
 *   for the near-null fields of the large one, and refinement stalls or diverges. */
enum { CD_PREC_FP64 = 0, CD_PREC_FP32_IR = 1 };

/* Preconditioner of the Krylov solve.
 * CD_PC_NONE: plain CG (the "CG" column of Tables 1-4, Section 6.2).
 * CD_PC_FD_D: exact inverse of the block diagonal D = blockdiag(A^(c,c)) of
 *   eq:diag by Kronecker fast diagonalisation (generalized eigenbasis of (S, M)).
 * CD_PC_FD_T: inverse of T = I_d (x) T_m(m_{p-1}) (x) ... of eq:kron_precond,
 *   by fast diagonalisation of the 1D factor.
 * CD_PC_MG: one V-cycle of the Galerkin multigrid of Section 6.1 (block
 *   prolongator eq:2by2prol, R = P^T, A_{l+1} = P^T A_l P) with a parallel
 *   smoother; the outer Krylov method is then flexible CG.
 * CD_PC_T_BAND: the same T^{-1} as CD_PC_FD_T, by banded Cholesky solves of the
 *   1D factor along every axis (Section 6.1 applies T by banded factorisation):
 *   O(N p) work per application instead of O(N m); p <= 6.
 * CD_PC_MIM: P_MIM of Section 6.2, the multi-iterative method as the preconditioner of
 *   (flexible) CG: two V-cycles from zero per application, each with the parallel smoother on
 *   every level and, at the finest level, p post-smoothing iterations of right-preconditioned
 *   GMRES with T (eq:kron_precond, banded solves) in place of the parallel post-smoother
 *   (Section 6.1); p <= 6.
 * CD_PC_WL: P_WL of Section 6.2: one V-cycle of the same multigrid applied to the block
 *   diagonal D = blockdiag(A^(c,c)) of eq:diag (coarse levels P^T D P, coarsest D inverted),
 *   with p PCG iterations preconditioned by T as the finest level's post-smoother; p <= 6. */
enum { CD_PC_NONE = 0, CD_PC_FD_D = 1, CD_PC_FD_T = 2, CD_PC_MG = 3, CD_PC_T_BAND = 4,
       CD_PC_MIM = 5, CD_PC_WL = 6 };

typedef struct {
  int precision;      /* CD_PREC_*                      (default CD_PREC_FP32_IR) */
  int precond;        /* CD_PC_*                        (default CD_PC_FD_D)      */
  int maxit;          /* max Krylov iterations in total (default 20000)          */
  double rtol;        /* stop when ||b - A x||_2 / ||b||_2 <= rtol (default 1e-10) */
  int max_batch;      /* RHS capacity of one call       (default 64)             */
  double inner_rtol;  /* FP32-IR: inner relative tolerance (default 1e-5)         */
  int inner_maxit;    /* FP32-IR: inner iteration cap per refinement step (4000)  */
  int max_outer;      /* FP32-IR: refinement steps before giving up (default 30)  */
  int smoother_degree;/* MG: Chebyshev smoothing steps per visit (default 2)      */
  int mg_m_min;       /* MG: stop coarsening at m <= mg_m_min and invert the
                          coarsest level densely (default 0: 16 for CD_PC_MG in
                          2D, else 3)                                            */
  int use_graphs;     /* capture the Krylov iteration in CUDA graphs (default 1)  */
  int chunk;          /* iterations per graph launch / host convergence poll (8)  */
  double mixed_switch_ratio; /* FP32-IR: parameter ratio above which the inner
                                Krylov solve is FP64 (default 1e4)                 */
  int fd_tensor_cores; /* FP32 FD transforms on tcgen05 (TF32 operands, FP32
                          accumulation; the Krylov method is then flexible) (1)   */
  int autotune;        /* time the FP32 2D apply kernels (folded-stencil tiles and two
                          tilings of the packed-pair kernel) and the 3D apply designs
                          for this shape at cd_create and keep the fastest (1).  The
                          kernels agree to FP32 rounding, not bit for bit, so a solve's
                          last bits can depend on the choice, which is made once per
                          (precision, m, p) and process (solves stay bit-identical
                          within it)                                               */
  int ext_residual;    /* 1 (default): the outer loop keeps the solution as an unevaluated
                          sum x_hi + x_lo of two FP64 vectors and evaluates b - A x in
                          double-FP64 arithmetic (about 106 significant bits), so the stopping
                          rule is not limited by FP64 rounding of A x (at beta/alpha = 1e+-6
                          and n = 256 an FP64 evaluation bottoms out near 1e-8).  0: FP64
                          solution and residual.                                           */
  int emulated_fp64;   /* 1 (default, with ext_residual and CD_PREC_FP32_IR): the FP64 inner
                          Krylov solves (2D and 3D) apply the operator in double-FP32 (about 48
                          significant bits) on the FP32 pipe, several times the FP64 rate on
                          GB300; their inner tolerance is then floored at 1e-6 relative and the
                          double-FP64 outer residual restores the accuracy.  0: FP64 applies.  */
  int reserved[4];
} cd_options;

typedef struct {
  int iters_outer;    /* refinement steps (1 for CD_PREC_FP64)                  */
  int iters_inner;    /* Krylov iterations summed over refinement steps         */
  double relres;      /* final ||b - A x|| / ||b|| of the solution the call returns
                         (cd_solve: x; cd_solve_ext: x + x_lo), evaluated in double-FP64
                         when ext_residual is set, else in FP64                    */
  double seconds;     /* wall time of the call (whole batch)                    */
  int status;         /* cd_status of this right-hand side: CD_OK iff relres <= rtol */
  double relres_hi;   /* the same for x alone (equal to relres for cd_solve)    */
} cd_result;

/* Fills *opt with the defaults listed above. */
CD_API void cd_default_options(cd_options* opt);

/* d * (n + p - 2)^d, the number of unknowns of one right-hand side (Section 5.1);
 * 0 for invalid arguments. */
CD_API size_t cd_dofs(int d, int p, int n);

CD_API const char* cd_strerror(cd_status s);
/* Text of the last CUDA / argument error seen by this thread ("" if none). */
CD_API const char* cd_last_error(void);

/* Builds a solver for (d, p, n): 1D B-spline mass / advection / stiffness bands
 * (eq:matr_M, eq:matr_A, eq:matr_S, Gauss-Legendre quadrature, FP64), the
 * multigrid hierarchy, the FD eigenbases (when the preconditioner needs them) and
 * the workspace for opt->max_batch right-hand sides.  alpha, beta are the
 * defaults used when a call passes NULL parameter arrays.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  opt == NULL selects defaults. */
CD_API cd_status cd_create(cd_solver* out, int d, int p, int n, double alpha,
                           double beta, const cd_options* opt, void* cuda_stream);

/* cd_create for an anisotropic mesh (Section 5: n_l = nu_l n intervals along x_l, the
 * spline space the tensor product of the 1D spaces of each direction).  n[0..d-1] are
 * the per-direction interval counts (host array of d ints, read during the call), so
 * component c has m_1 ... m_d unknowns, m_l = n[l] + p - 2, and a right-hand side is
 * [d][m_1]...[m_d] (x_d fastest), d prod_l m_l doubles.  The operator is eq:matr_Amu /
 * eq:matr_Amu3D with the 1D matrices of direction l in the l-th Kronecker position.
 * Offered: cd_apply, cd_apply_f32, cd_solve, cd_solve_ext, cd_solve_host, cd_lanczos
 * and cd_precond, with precond CD_PC_NONE or CD_PC_FD_D (fast diagonalisation of the
 * block diagonal with each direction's generalized eigenbasis); the residual is
 * evaluated in FP64 (ext_residual, emulated_fp64, fd_tensor_cores and autotune are
 * ignored: the handle uses one banded pass per direction and SIMT FD transforms).
 * opt == NULL selects defaults with CD_PC_NONE.  CD_EINVAL for d not 2 or 3, p < 1,
 * n NULL, any m_l < 2, d prod m_l >= 2^31, a bad parameter, or another precond; the
 * multigrid entry points (cd_levels returns 0, cd_restrict, cd_prolong, cd_get_bands,
 * cd_get_eig) reject such a handle. */
CD_API cd_status cd_create_aniso(cd_solver* out, int d, int p, const int* n, double alpha,
                                 double beta, const cd_options* opt, void* cuda_stream);
CD_API cd_status cd_destroy(cd_solver h);

/* y = A w for nrhs right-hand sides (matrix-free, sum-factorised; eq:matr_Amu /
 * eq:matr_Amu3D).  Device pointers, FP64 / FP32 respectively. */
CD_API cd_status cd_apply(cd_solver h, const double* w, double* y, int nrhs,
                          const double* alphas, const double* betas);
CD_API cd_status cd_apply_f32(cd_solver h, const float* w, float* y, int nrhs,
                              const double* alphas, const double* betas);

/* Solves A x = b (eq:system) for nrhs right-hand sides from x_0 = 0 with the
 * handle's options; stop rule ||b - A x|| / ||b|| <= rtol (Section 6.2 with the
 * handle's tolerance).  b, x: device FP64.  res: nrhs host entries (may be NULL).
 * Returns the worst per-RHS status. */
CD_API cd_status cd_solve(cd_solver h, const double* b, double* x, int nrhs,
                          const double* alphas, const double* betas, cd_result* res);

/* As cd_solve, returning the solution as the unevaluated sum x + x_lo of two FP64 vectors
 * (x = the FP64 rounding of the sum; x_lo: device FP64, same layout, may be NULL).  With
 * ext_residual set, the refinement loop of Section 6.2's stopping rule measures
 * ||b - A (x + x_lo)|| in double-FP64, so the rule can be met where an FP64 vector cannot
 * represent a solution that accurate (at beta/alpha = 1e+-6 the exact solution rounded to FP64
 * has a relative residual near 1e-10 at n = 256).  res[i].relres is that of x + x_lo and
 * res[i].relres_hi that of x alone.  Without ext_residual x_lo is filled with zeros. */
CD_API cd_status cd_solve_ext(cd_solver h, const double* b, double* x, double* x_lo, int nrhs,
                              const double* alphas, const double* betas, cd_result* res);

/* As cd_solve with host b and x (pageable or pinned): copies b to the device,
 * solves, copies x back; all three steps are inside the call. */
CD_API cd_status cd_solve_host(cd_solver h, const double* b_host, double* x_host,
                               int nrhs, const double* alphas, const double* betas,
                               cd_result* res);

/* One application z = B^{-1} r of a preconditioner kind (CD_PC_FD_D: D^{-1},
 * eq:diag; CD_PC_FD_T and CD_PC_T_BAND: T^{-1}, eq:kron_precond; CD_PC_MG: one
 * V-cycle from zero) in FP64 (`f32` = 0) or FP32 (`f32` = 1, pointers then hold
 * floats).  r, z: device pointers, nrhs right-hand sides in the layout above;
 * r and z may not overlap.  The data a kind needs is built on its first use
 * (the eigenbases for the FD kinds, the banded factor for CD_PC_T_BAND; the
 * multigrid hierarchy exists from cd_create).  CD_EINVAL for an unknown kind,
 * CD_PC_T_BAND with p > 6, or the argument errors listed at the top. */
CD_API cd_status cd_precond(cd_solver h, int kind, const void* r, void* z, int nrhs,
                            const double* alphas, const double* betas, int f32);

/* Copies the library's 1D bands of multigrid level `level` (0 = finest) to host
 * arrays of m_l * (2P+1) doubles each, row i holding X(i, i-P .. i+P):
 * M, A (advection, stored exactly skew), S.  *m_out = m_l, *P_out = P.
 * Any of M, A, S may be NULL to only query the sizes. */
CD_API cd_status cd_get_bands(cd_solver h, int level, double* M, double* A, double* S,
                              int* m_out, int* P_out);

/* Host-only set-up queries (no handle, no GPU; the library's own FP64 host code).
 * cd_setup_bands: the 1D bands of Section 3.2 for degree p on n intervals (Gauss-Legendre
 *   quadrature, p + 1 points per interval, Dirichlet basis, m = n + p - 2), Galerkin-coarsened
 *   `level` times with the 3-tap prolongator of Section 6.1 (P^T X P); layout as
 *   cd_get_bands (before a handle replaces the interior rows by the central row).
 * cd_setup_eig: as cd_get_eig for the finest grid of (p, n).
 * cd_setup_tband: the banded Cholesky factor T_m(m_{p-1}) = L L^T (eq:kron_precond,
 *   half-bandwidth q = p - 1) used by CD_PC_T_BAND: Lb[(m + q) * q] with
 *   Lb[i*q + t] = L(i, i-q+t) (zero left of column 0 and in the q rows past m), and
 *   dinv[m] = 1 / L(i, i).
 * All three: CD_EINVAL unless 1 <= p <= 6, n >= 1, m >= 1 (and level within the grid
 * hierarchy); caller-owned host output arrays, any of which may be NULL. */
CD_API cd_status cd_setup_bands(int p, int n, int level, double* M, double* A, double* S,
                                int* m_out, int* P_out);
CD_API cd_status cd_setup_eig(int p, int n, int which, double* U, double* lam);
CD_API cd_status cd_setup_tband(int p, int n, double* Lb, double* dinv);

/* Number of multigrid levels of the handle. */
CD_API int cd_levels(cd_solver h);

/* Copies an FD eigenbasis to host: which = 0: S U = M U diag(lam), U^T M U = I
 * (generalized, for D); which = 1: T_1 U = U diag(lam), U^T U = I (for T).
 * U: m*m doubles, row-major U[i*m + k] = entry (i, k), columns = eigenvectors,
 * lam ascending. */
CD_API cd_status cd_get_eig(cd_solver h, int which, double* U, double* lam);

/* Multigrid transfer between level l and l+1 (eq:2by2prol), FP64 device:
 * cd_restrict: coarse = P^T fine; cd_prolong: fine += P coarse. */
CD_API cd_status cd_restrict(cd_solver h, int level, const double* fine, double* coarse,
                             int nrhs);
CD_API cd_status cd_prolong(cd_solver h, int level, const double* coarse, double* fine,
                            int nrhs);

/* ---------------------------------------------------------------- spectral validation
 * Eigenvalue functions of the d x d symbol f^{p,alpha,beta} of Theorem 5.1 (eq:f2D, d = 2) /
 * Theorem 5.5 (eq:f3D, d = 3), sampled on the grid Gamma of Section 5.3: theta_k = k pi / mg,
 * k = 1..mg per direction, points in C order (theta_1 slowest).  lam: device, mg^d * d doubles,
 * the d eigenvalues of each point in ascending order (Lambda_1..Lambda_d of Section 5.3).
 * lap: device, mg^d doubles or NULL, the Laplacian symbol (eq:lapl2D / eq:lapl3D) that bounds
 * them, min(alpha,beta) lap <= lambda_i <= max(alpha,beta) lap (Theorems 5.2 / 5.6).
 * nu: d host doubles (the anisotropy n_l = n nu_l of the theorems' weights gamma_i, delta_i) or
 * NULL for nu = 1.  Stream-ordered on `cuda_stream`; nothing is allocated.  CD_EINVAL for d not
 * in {2,3}, p outside 1..8, mg < 1, non-positive parameters or weights, lam == NULL. */
CD_API cd_status cd_symbol_eigs(int d, int p, double alpha, double beta, const double* nu,
                                int mg, double* lam, double* lap, void* cuda_stream);

/* `steps` Lanczos steps with the handle's FP64 operator (eq:matr_Amu / eq:matr_Amu3D) from the
 * start vectors v0 (device, nrhs right-hand-side layout, any nonzero vectors), no
 * reorthogonalisation: lam_min / lam_max (host, nrhs) receive the extreme eigenvalues of the
 * Lanczos tridiagonal matrix (Ritz values, inside [lambda_min(A), lambda_max(A)] and converging
 * to them), the check of Section 5.3's spectra against the symbol bounds.  diag / offdiag (host,
 * nrhs * steps each, or NULL) receive alpha_j and beta_{j+1}.  A solve whose Krylov space becomes
 * invariant stops early (its remaining coefficients are zero).  CD_EINVAL for steps outside
 * 1..4096 or the argument errors listed at the top. */
CD_API cd_status cd_lanczos(cd_solver h, const double* v0, int nrhs, int steps,
                            const double* alphas, const double* betas, double* lam_min,
                            double* lam_max, double* diag, double* offdiag);

/* Number of this library's kernels launched by this process so far. */
CD_API uint64_t cd_kernel_launches(void);

/* ---------------------------------------------------------------- serving runtime
 * Continuous batching of solve requests (the paper has no serving layer; this runs the
 * solves of eq:system for many independent requests on one GPU).  Requests of one shape
 * (d, p, n) share a cached solver whose `max_batch` right-hand-side slots run as a session:
 * each slot follows the refinement loop of cd_solve on its own schedule, one chunk of Krylov
 * iterations (cd_options.chunk) per step.  A pool of `workers` threads, each stepping one
 * shape at a time on that shape's stream, takes the shape that is due (its last step or its
 * oldest queued request is oldest), admits queued requests into free slots (all right-hand
 * sides of a request together), runs one step and completes the slots that finished: requests
 * join and leave between chunks of iterations while the other slots keep running, and
 * different shapes step concurrently.  A shape's solver is admitted when its device footprint
 * fits in `hbm_budget`, evicting idle solvers (least recently used) when needed.  A request's
 * results do not depend on what else runs (every kernel is masked per slot and every
 * reduction has a fixed order per slot): they equal those of cd_solve_host on the same
 * right-hand side with half the tolerance.  The server returns the FP64 vector x, whose
 * residual exceeds that of the refinement's x + x_lo by the rounding of x (about
 * eps |A| |x|, a sizeable part of 1e-10 at beta/alpha near 1e+-6): the sessions refine to
 * solve.rtol / 2 and a right-hand side's status is CD_OK iff the returned x has relres <=
 * solve.rtol.  Host buffers only; the server copies b at submit and x at poll/wait. */
typedef struct cd_server_s* cd_server;

typedef struct {
  size_t hbm_budget;  /* device bytes the cached solvers may hold (0: 80% of free memory) */
  int workers;        /* shapes stepped concurrently, one thread each (default 8)          */
  int max_batch;      /* session slots (right-hand sides in flight) per shape (default 16) */
  double timeout_s;   /* a request still queued after this many seconds fails with
                         CD_TIMEOUT (0: no limit)                                           */
  cd_options solve;   /* options of every solve (default: cd_default_options, CD_PC_MG)    */
} cd_server_options;

typedef struct {
  uint64_t submitted, completed, failed, batches, solves; /* batches = session steps,
                                                            solves = right-hand sides     */
  double p50_s, p99_s;  /* latency (submit to completion) of completed requests           */
  double mean_batch;    /* occupied slots per session step                                */
  double solves_per_s;  /* right-hand sides solved / (last completion - first submit)     */
  size_t bytes_in_use;  /* estimated device bytes of the cached solvers                   */
  int handles;          /* cached solvers                                                 */
} cd_server_stats;

CD_API void cd_server_default_options(cd_server_options* opt);
/* Starts the worker threads on the current CUDA device. */
CD_API cd_status cd_server_create(cd_server* out, const cd_server_options* opt);
/* Queues a request: nrhs right-hand sides (host, layout as above) with per-RHS alphas /
 * betas (host arrays of nrhs).  CD_EINVAL for a bad shape, parameters or nrhs > max_batch. */
CD_API cd_status cd_server_submit(cd_server s, int d, int p, int n, const double* alphas,
                                  const double* betas, const double* b_host, int nrhs,
                                  uint64_t* ticket);
/* Non-blocking: *done = 0 while the request runs; when done, copies x (nrhs * cd_dofs
 * doubles, may be NULL) and res (nrhs entries, may be NULL), releases the ticket and returns
 * the request's worst status. */
CD_API cd_status cd_server_poll(cd_server s, uint64_t ticket, double* x_host, cd_result* res,
                                int* done);
/* Blocking form of cd_server_poll (timeout_s <= 0: no limit; CD_TIMEOUT if it expires, the
 * ticket then stays valid). */
CD_API cd_status cd_server_wait(cd_server s, uint64_t ticket, double* x_host, cd_result* res,
                                double timeout_s);
/* Cancels a request that has not been admitted into slots (it completes with CD_CANCELLED);
 * CD_EINVAL if it is already on the GPU or unknown. */
CD_API cd_status cd_server_cancel(cd_server s, uint64_t ticket);
CD_API cd_status cd_server_stats_get(cd_server s, cd_server_stats* out);
/* Stops the workers after their current steps and frees every cached solver. */
CD_API cd_status cd_server_destroy(cd_server s);

/* y = A w for d = 3 (FP64 device vectors, layout as above, one (alpha, beta) for all
 * nrhs right-hand sides), without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc -- code
 * that runs inside a host framework whose allocator owns all device memory and forbids
 * side allocations, or latency-critical paths that cannot accept the implicit device
 * synchronisation of cudaMalloc / cudaFree.  It computes the same product as cd_apply
 * on a handle created for (3, p, n) with the same kernels, but needs no handle.
 *
 * Its working memory is a fixed 48 MiB array in the library's device image: every GPU
 * that loads the library holds it until the process exits.  A call needs about
 * 18 m^3 nrhs + 3 m (2p+1) + 2 nrhs doubles of it (m = n + p - 2; for one right-hand
 * side m <= 70); larger requests return CD_EINVAL with the limit in cd_last_error().
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  The address
 * is kept per device and looked up again if the device's context was rebuilt (a
 * cudaDeviceReset).  Every call shares the array and overwrites what it reads, so calls
 * whose work overlaps on the GPU (on different streams or from different threads) race.
 * The call copies the 1D bands and parameters from host memory to the array with
 * cudaMemcpyAsync on `cuda_stream` (NULL = legacy default stream), then launches the
 * three banded FP64 passes on it; it does not wait for the GPU. */
CD_API cd_status cd_apply3d_static(int p, int n, double alpha, double beta, const double* w,
                                   double* y, int nrhs, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CURLDIV_H */
