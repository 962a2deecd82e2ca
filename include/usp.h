/*
 * usp.h -- C ABI of the GB300 (sm_103a) solver for the fixed-point
 * (Richardson) iteration with the universal split preconditioner
 * (Vettenburg & Vellekoop, "A universal matrix-free split preconditioner for
 * the fixed-point iterative solution of non-symmetric linear systems").
 *
 * The problem is a canonical linear system A x = y with A = L + V (Sec. 2):
 *   - L is translation invariant on a periodic grid, given by its Fourier
 *     symbol  Lhat(p) = a |p|^2 + b,  p = 2 pi m / (n dx), m the FFT-order
 *     frequency index on each axis;
 *   - V is a pointwise potential with max |V| < 1;
 *   - A is accretive (Eq. accretivity-condition).
 * The solver runs Algorithm 1 on the forward-eliminated operator (Sec. 2.1)
 *     Delta = B[(L+I)^-1 (B x + y) - x],   B = I - V,
 *     x     = x + alpha Delta,
 * until ||Delta|| / ||B (L+I)^-1 y|| < tol, with (L+I)^-1 applied as an FFT,
 * a pointwise multiply by 1/(Lhat+1) and an inverse FFT (Eq.
 * laplacian_inverse).  All arithmetic of the iteration is FP32 on the GPU;
 * norms are summed in FP64; the refinement residual y - A x is formed in
 * double-float (pairs of FP32 values, 48-bit significand) or FP64.
 *
 * Conventions for every entry point:
 *   - Fields are C-contiguous, last axis fastest ([n0][n1][n2]); complex
 *     fields are complex64 (two interleaved float32: re, im), 8-byte aligned
 *     (16-byte aligned recommended).  A real potential is float32.
 *   - "device pointer" = memory the GPU can address (cudaMalloc, torch CUDA
 *     tensors); "host pointer" = ordinary (pinned or pageable) CPU memory.
 *   - Every call returns a usp_status; no call aborts or throws.  On error
 *     the outputs are unspecified unless stated; usp_last_error() gives a
 *     one-line description of the last failure on the calling thread.
 *   - Calls on one solver handle must not overlap in time (a handle is not
 *     thread-safe); separate handles are independent.
 */
#ifndef USP_H
#define USP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  USP_OK = 0,
  USP_ERR_INVALID_ARG = 1,       /* null pointer, bad ndim, tol < 0, ...      */
  USP_ERR_UNSUPPORTED_SIZE = 2,  /* an axis length is not supported (below)   */
  USP_ERR_V_NOT_CONTRACTIVE = 3, /* max |V| >= 1 (Thm 1 needs ||V|| < 1)      */
  USP_ERR_NOT_ACCRETIVE = 4,     /* Re(Lhat(p) + 1) <= 0 for some p (L+I not
                                    invertible / A + B not accretive,
                                    Corollary)                                */
  USP_ERR_ALPHA_RANGE = 5,       /* alpha not finite or outside (0, 2]        */
  USP_ERR_NOT_CONVERGED = 6,     /* maxit reached, or stagnation without
                                    refinement; x holds the last iterate      */
  USP_ERR_DIVERGED = 7,          /* ||Delta|| grew fourfold above its first
                                    value: the contraction (Thm 1) does not
                                    hold for these inputs                     */
  USP_ERR_NONFINITE = 8,         /* NaN/Inf in V, y, x0 or an iterate         */
  USP_ERR_CUDA = 9,              /* a CUDA runtime call failed                */
  USP_ERR_OOM = 10               /* device allocation failed                  */
} usp_status;

/* Grid: ndim in {1,2,3}; n[0..ndim-1] axis lengths, n[ndim-1] fastest;
 * each a power of two in [2, 256], or 96, 192, 384 (3 * 2^k) or 512 (the
 * transforms add a radix-3 or radix-2 outer stage).  dx > 0 is the grid
 * spacing (all axes). */
typedef struct {
  int32_t ndim;
  int64_t n[3];
  double dx;
} usp_grid;

/* Fourier symbol of L (Sec. 2: L translation invariant, so F L F^-1 is a
 * multiplication by Lhat(p)).
 * USP_LSYM_QUADRATIC (kind 0, the default of a zero-initialised struct):
 *   Lhat(p) = a |p|^2 + b  (complex a, b).
 *   Helmholtz (Sec. 3.1, Eq. laplacian_inverse): a = -1/c, b = kbar2/c.
 *   Diffusion (Sec. 3.2, scalar D, steady state): a = D/c, b = etabar/c.
 * USP_LSYM_TABLE (kind 1): Lhat given point by point in k-space: `table`
 *   is a device pointer to N complex64 values in the grid's layout (C order,
 *   last axis fastest), entry (m0, m1, m2) for the FFT-order frequency
 *   indices m_ax (0 .. n_ax - 1; index m stands for m or m - n_ax).  Any
 *   translation-invariant L (a finite-difference Laplacian, anisotropic or
 *   dispersive operators) fits.  Copied at create; Re(Lhat + 1) > 0 and
 *   finiteness are checked there.  Single-problem solvers only (batches and
 *   usp_solve_noalloc take the quadratic kind); a, b are ignored. */
typedef enum { USP_LSYM_QUADRATIC = 0, USP_LSYM_TABLE = 1 } usp_lsym_kind;

typedef struct {
  double a_re, a_im;
  double b_re, b_im;
  int32_t kind;        /* usp_lsym_kind */
  const void* table;   /* USP_LSYM_TABLE: device, N complex64 */
} usp_lsymbol;

/* Outcome of a solve (valid for USP_OK and USP_ERR_NOT_CONVERGED). */
typedef struct {
  int32_t iterations;        /* Delta evaluations, all phases together     */
  int32_t converged;         /* 1 if the last ||Delta||/ref_norm < tol      */
  int32_t refinements;       /* residual restarts performed (refinement)    */
  int32_t stagnated;         /* 1 if the FP32 iteration stopped improving  */
  double final_rel_residual; /* last ||Delta|| / ref_norm                   */
  double ref_norm;           /* ||B (L+I)^-1 y||, the alpha-free
                                ||Gamma^-1 y|| of Algorithm 1's test        */
  double alpha;              /* step size used                              */
} usp_result;

/* Solver options (usp_solver_set_options).  Zero-initialised = defaults. */
typedef struct {
  /* 0: refinement on (default) -- when the FP32 iteration reaches 8*tol or
   *    stops improving, y - A x is formed in double-float (or FP64, see
   *    residual_fp64) and the same FP32
   *    iteration continues on the correction z with source y - A x, which
   *    has exactly the same Delta (A + B = L + I, Sec. 2.1); x = x + z.
   * 1: plain -- Algorithm 1 exactly: stop at tol or maxit.                 */
  int32_t plain;
  /* 0: automatic (on-chip where it applies, except batches of 192^2 and
   *    256^2 problems whose clusters do not all fit on the device at once;
   *    split-y for single 3-D problems nz x 256 x 256 unless tc_dft or
   *    no_tma is set; else pencil);
   * 1: pencil schedule (one FFT axis per pass);
   * 2: fused 3-D schedule (two passes per iteration; 3-D grids nz x 256 x
   *    256, single problem);
   * 3: on-chip schedule (square 2-D grids n x n, n in {32, 64, 96, 128,
   *    192, 256}):
   *    each problem's fields stay in the shared memory of one thread-block
   *    cluster and one launch runs a whole phase of iterations;
   * 4: split-y schedule (single 3-D problems nz x 256 x 256, nz in {32, 64,
   *    128, 256}): two passes per iteration; the 256-point y transform is
   *    split 16 x 16 between a rows pass (x transform and one 16-point
   *    stage, tiles of 16 rows of one plane) and a column pass (the other
   *    16-point stage, z transform, spectral multiply); 64 bytes per point
   *    per iteration.                                                       */
  int32_t schedule;
  /* iterations per CUDA-graph launch between convergence polls; 0: auto   */
  int32_t chunk;
  /* maximum refinements per solve; 0: default (4)                          */
  int32_t max_refinements;
  /* 1: strided-axis passes load and store with plain global accesses
   *    instead of TMA-staged tiles (for comparison); 0: TMA (default)      */
  int32_t no_tma;
  /* columns per staged strided-axis tile: 8, 16 or 32 (4, 2 or 1 CTAs
   * per SM), or 0 for the library's default                                */
  int32_t cols_tile;
  /* 1: the 256-point transforms of the strided-axis passes run on the
   *    tensor cores (tcgen05, TF32 split into three products for FP32-level
   *    accuracy; single problems, pencil schedule); 0: CUDA cores           */
  int32_t tc_dft;
  /* rows (and k-space columns) per CTA of the on-chip schedule: 16, or 8
   * (n <= 128; twice the CTAs per problem), or 0 for the library's choice */
  int32_t onchip_rows;
  /* testing hook, 0 in normal use: nonzero makes the on-chip schedule's
   * first exchange expect bytes that are never sent, with a short wait
   * limit, so the solve ends with the bounded-wait error (USP_ERR_CUDA,
   * "timed out") and the solver stays usable                               */
  int32_t test_wait_fault;
  /* arithmetic of the refinement residual y - A x (and of usp_apply_A and
   * usp_residual): 0 (default) double-float -- each real number the
   * unevaluated sum of two FP32 values, a 48-bit significand, built from
   * exact two-sum / two-product steps; several times faster than FP64 on a
   * GPU whose FP64 rate is a small fraction of its FP32 rate; 1: FP64.
   * Both carry the residual far below the FP32 iteration's own floor.     */
  int32_t residual_fp64;
} usp_options;

typedef struct usp_solver usp_solver;

/* Create a solver for one operator A = L + V.
 *   grid, lsym : see above (host pointers, copied).
 *   V          : device pointer, N = prod(n) complex64 values, or float32
 *                values if V_is_real != 0.  Copied into solver-owned device
 *                memory before return; the caller may free it afterwards.
 *   alpha      : step size; <= 0 selects alpha = Re[B^-1] = min_r Re
 *                1/(1 - V(r)), the worst-case optimum of the
 *                convergence-rate theorem (appendix).  alpha in (0, 1] is
 *                always safe (Corollary).
 *   cuda_stream: cudaStream_t the caller orders work on (0 = legacy
 *                default stream).  Solves wait for work already queued on it.
 * Validation (Sec. 2, Thm 1, Corollary): max |V| < 1, V finite,
 * Re(Lhat(p) + 1) > 0 on the grid.  Allocates the solver's device memory
 * (V copy, one scratch field, reduction buffers).  On success *out owns the
 * solver; release it with usp_solver_destroy. */
usp_status usp_solver_create(const usp_grid* grid, const usp_lsymbol* lsym,
                             const void* V, int32_t V_is_real, double alpha,
                             void* cuda_stream, usp_solver** out);

/* ---- batches of problems on one grid --------------------------------------
 *
 * `count` independent problems A_j = L_j + V_j on the same grid, solved
 * together: every pass of Algorithm 1 (Sec. 2.1) runs once over all problems,
 * each with its own symbol, step, convergence test, residual history and
 * refinement.  The paper solves one problem at a time; the batch is this
 * library's throughput form of the same iteration, and each problem follows
 * exactly the path it would take alone.
 *   lsyms, alphas: host arrays of `count` (alphas[j] <= 0: automatic).
 *   V: device pointer, count * N values (problem j at offset j * N), complex64
 *      or float32 (V_is_real, one setting for the whole batch).
 * count >= 1; count > 1 needs a 2-D or 3-D grid whose number of lines along
 * the last axis per problem, N / n_last, is a multiple of 256 * m / n_last
 * with m = 2^ceil(log2(n_last) / 2) (16 lines for n_last = 256, 32 for 64
 * and 128), so that no block of the line passes straddles two problems
 * (USP_ERR_UNSUPPORTED_SIZE otherwise).  Validation as usp_solver_create, for every problem.  A batch
 * solver is solved with usp_batch_solve (usp_solve and usp_solve_host
 * return USP_ERR_INVALID_ARG); usp_apply_A, usp_residual and usp_time_passes
 * act on the whole batch (usp_residual's rel_out is over all problems). */
usp_status usp_batch_create(const usp_grid* grid, int32_t count,
                            const usp_lsymbol* lsyms, const void* V,
                            int32_t V_is_real, const double* alphas,
                            void* cuda_stream, usp_solver** out);

/* Algorithm 1 for every problem of a batch solver.  y, x: device pointers,
 * count * N complex64 (layout as V).  ref_norms: host array of count (<= 0:
 * automatic) or NULL (all automatic).  results, statuses: host arrays of
 * count, or NULL; statuses[j] is what usp_solve would return for problem j
 * alone.  Returns USP_OK when every problem converged, else the status of
 * the lowest-numbered problem that did not (its message in usp_last_error).
 * Synchronous. */
usp_status usp_batch_solve(usp_solver* s, const void* y, void* x,
                           int32_t use_x0, double tol, int32_t maxit,
                           const double* ref_norms, usp_result* results,
                           usp_status* statuses);

/* Residual history of problem `problem` of the last solve (as
 * usp_residual_history, which reports problem 0). */
usp_status usp_batch_history(const usp_solver* s, int32_t problem,
                             double* host_out, int32_t capacity,
                             int32_t* n_out);

/* Solve several solvers (single problems or batches, any grids) at the same
 * time: one host thread per solver drives that solver's own stream, so their
 * passes run concurrently on the GPU -- the form for many problems of
 * different sizes (one batch solver per size).  Each solver runs
 * usp_batch_solve (Algorithm 1 per problem, automatic reference norms) on
 * (ys[i], xs[i]) (device pointers, layout as for that solver).  results,
 * statuses: host arrays over all problems, solver by solver, or NULL.
 * Returns USP_OK when every problem converged, else the first failing
 * solver's status and message.  A solver may appear only once. */
usp_status usp_solve_many(usp_solver* const* solvers, int32_t count,
                          const void* const* ys, void* const* xs,
                          int32_t use_x0, double tol, int32_t maxit,
                          usp_result* results, usp_status* statuses);

/* Replace the options of a solver (host pointer, copied). */
usp_status usp_solver_set_options(usp_solver* s, const usp_options* opt);

/* Algorithm 1 (Sec. 2.1).
 *   y       : device pointer, N complex64, the canonical source (borrowed
 *             for the duration of the call, not modified).
 *   x       : device pointer, N complex64.  In: the initial estimate if
 *             use_x0 != 0 (otherwise ignored, the iteration starts at 0).
 *             Out: the last iterate.
 *   tol     : stop when ||Delta_i|| / ref_norm < tol (tol >= 0; 0 runs
 *             exactly maxit iterations in plain mode).
 *   maxit   : iteration limit (>= 1), counted over all refinement phases.
 *   ref_norm: > 0 uses this denominator (e.g. to resume a solve); <= 0
 *             computes ||B (L+I)^-1 y|| (one extra FFT pair if use_x0).
 * Returns USP_OK when converged, USP_ERR_NOT_CONVERGED when maxit is hit
 * or the plain FP32 iteration stagnates (x and *out still valid),
 * USP_ERR_NONFINITE / USP_ERR_DIVERGED on failure.  Synchronous: returns
 * after the GPU work finished.  *out may be NULL. */
usp_status usp_solve(usp_solver* s, const void* y, void* x, int32_t use_x0,
                     double tol, int32_t maxit, double ref_norm,
                     usp_result* out);

/* The same solve with host buffers: y_host (N complex64) is copied to the
 * device, the solve runs on solver-owned device buffers, and the result is
 * copied back into x_host (which also supplies x0 when use_x0 != 0).
 * Pinned host memory gives the fastest copies. */
usp_status usp_solve_host(usp_solver* s, const void* y_host, void* x_host,
                          int32_t use_x0, double tol, int32_t maxit,
                          double ref_norm, usp_result* out);

/* Residual history of the last solve: history[i] = ||Delta_{i+1}||/ref_norm
 * (Fig. 1d plots this quantity).  Copies min(capacity, count) values into
 * host_out (host pointer) and writes the count to *n_out. */
usp_status usp_residual_history(const usp_solver* s, double* host_out,
                                int32_t capacity, int32_t* n_out);

/* Forward operator A x = L x + V x (Sec. 2, the problem statement), in the
 * refinement residual's arithmetic on the GPU (double-float, or FP64 with
 * the residual_fp64 option), for the unpreconditioned residual ||A x - y||/||y||
 * of the paper's tables (Sec. 4.1).  x, Ax: device pointers, N complex64;
 * Ax may not alias x. */
usp_status usp_apply_A(usp_solver* s, const void* x, void* Ax);

/* r = y - A x, the refinement residual (double-float arithmetic, or FP64
 * with the residual_fp64 option); r is written as complex64 (device
 * pointer) and, if rel_out is not NULL, ||r||/||y|| (summed in FP64)
 * to *rel_out (host pointer).  r may be NULL when only the norm is wanted. */
usp_status usp_residual(usp_solver* s, const void* x, const void* y, void* r,
                        double* rel_out);

/* The step size the solver uses (host pointer out). */
usp_status usp_solver_alpha(const usp_solver* s, double* alpha_out);

/* Free all resources of a solver (NULL is ignored). */
void usp_solver_destroy(usp_solver* s);

/* Canonical form on the host, FP64 (Sec. 2.2 and 3.1).  Helmholtz problem
 * laplacian(psi) + k2(r) psi = -S(r):
 *   kbar2, rho = centre and radius of the smallest circle enclosing the
 *   values k2(r) (the smallest-circle problem; Welzl's algorithm);
 *   c = -rho/(0.95 i) scaled by norm_v: c = i rho / norm_v;
 *   V = (k2 - kbar2)/c, y = -S/c, a = -1/c, b = kbar2/c.
 * k2, S: host pointers to n complex128 values (interleaved doubles).
 * V_out, y_out: host pointers to n complex64 values (written).
 * lsym_out, c_out (2 doubles: re, im), bias_out (2 doubles): written.
 * norm_v in (0, 1) (the paper uses 0.95).  Returns USP_ERR_INVALID_ARG for
 * a homogeneous medium (rho = 0: c undefined). */
usp_status usp_canon_helmholtz(const double* k2, const double* S, int64_t n,
                               double norm_v, float* V_out, float* y_out,
                               usp_lsymbol* lsym_out, double* c_out,
                               double* bias_out);

/* Canonical form of steady diffusion -D laplacian(u) + eta(r) u = S(r)
 * (Sec. 3.2 with scalar constant D): etabar, rho = midpoint and half-range
 * of eta; c = rho / norm_v (real, positive); V = (eta - etabar)/c (real),
 * y = S/c, a = D/c, b = etabar/c.
 * eta: host, n doubles.  S: host, n complex128.  V_out: host, n float32.
 * y_out: host, n complex64.  c_out: 1 double. */
usp_status usp_canon_diffusion(const double* eta, double D, const double* S,
                               int64_t n, double norm_v, float* V_out,
                               float* y_out, usp_lsymbol* lsym_out,
                               double* c_out, double* bias_out);

/* ---- allocation-free solve (no counterpart in the paper) ----------------
 *
 * For callers that cannot allocate device memory -- e.g. a process whose
 * device memory was handed to another allocator at start-up, or a hot loop
 * that must not call cudaMalloc/cudaFree because they synchronise the
 * device.  Runs the plain fixed-point iteration of this library (FP32, no
 * refinement), starting from x = 0, on the caller's V, y and x, with
 * all scratch (one field, partial sums, state, residual history) in a fixed
 * area of USP_NOALLOC_BYTES compiled into the library.  Grids: each axis a
 * power of two in [2, 256], at most USP_NOALLOC_MAX_POINTS points in all;
 * quadratic symbol only (USP_LSYM_QUADRATIC); maxit up to
 * USP_NOALLOC_MAX_ITERS.  Other axis lengths (96, 192, 384, 512) and larger
 * grids return USP_ERR_UNSUPPORTED_SIZE, a tabulated symbol or a larger
 * maxit USP_ERR_INVALID_ARG, each with a message (usp_last_error).  It calls
 * no allocation routine.
 *
 * The scratch area belongs to the library's device code, which CUDA may
 * load lazily: the area may then be reserved on a device only at the first
 * call there, not when the library is loaded.  A caller that hands its
 * device memory to another allocator should therefore make one call first
 * (a tiny grid will do); if the reservation fails, the call returns
 * USP_ERR_OOM.  Once reserved, the area stays with the device until the
 * process exits.
 *
 * The first call on a device also does a one-time set-up there (looks up
 * the scratch area's device address, uploads the FFT twiddle tables): make
 * that first call before any stream capture.  All calls share the one
 * scratch area, whose contents persist between calls (each call rewrites
 * what must start from zero); calls whose GPU work overlaps in time race on
 * it, so serialise them.  Other arguments as for usp_solver_create and
 * usp_solve (device pointers V, y, x; x is output only).  Synchronous. */
#define USP_NOALLOC_MAX_POINTS (1 << 19)
#define USP_NOALLOC_MAX_ITERS 65536
#define USP_NOALLOC_BYTES 4751872
usp_status usp_solve_noalloc(const usp_grid* grid, const usp_lsymbol* lsym, const void* V,
                             int32_t V_is_real, double alpha, const void* y, void* x,
                             double tol, int32_t maxit, void* cuda_stream, usp_result* out);

/* ---- block variants of the canonical form (Sec. 2.2, Sec. 3.2) ----------
 *
 * The same Algorithm 1 (forward-eliminated, Sec. 2.1) on an unknown with K
 * components per grid point, V a K x K matrix per point and L a K x K
 * matrix of Fourier multipliers.  Fields are K consecutive planes of N =
 * prod(n) complex64 values (component k at offset k N).  FP32 arithmetic,
 * norms in FP64; plain Algorithm 1 (no refinement).
 *
 * USP_VARIANT_ANTISYMMETRIC (Sec. 2.2, Eq. antisymmetrised), K = 2: for a
 *   raw problem A0 x0 = y0 that is not accretive, A = [[0, -A0^*], [A0, 0]]/c
 *   with real c; x = [x0; x0'] where x0' solves the adjoint problem.  Per
 *   point V = [[0, -conj(v)], [v, 0]]; per frequency L = [[0, -conj(l)],
 *   [l, 0]], l = a |p|^2 + b.  params = (a_re, a_im, b_re, b_im); V: device,
 *   N complex64 values v.  (usp_canon_antisymmetric builds them for the
 *   Helmholtz operator.)
 * USP_VARIANT_FLUX_DIFFUSION (Sec. 3.2, Eq. diffusion-equation-matrix-form
 *   with d/dt = 0, scalar D(r)), K = 1 + ndim: unknown C^1/2 [u; J], per
 *   point V = diag(Vu, VJ I), per frequency L + I = [[alpha, i s p^T],
 *   [i s p, beta I]].  params = (alpha, beta, s), alpha, beta >= 1 (L
 *   accretive); V: device, two planes of N float32 (Vu, then VJ).
 *   (usp_canon_flux_diffusion builds them.)
 * Validation: max over points of ||V|| < 1, V finite.  alpha <= 0 selects
 * min over points of Re 1/lambda over the eigenvalues lambda of B = I - V
 * (B is normal: 1/(1 + |v|^2) antisymmetric, 1/(1 - V) flux). */
typedef enum {
  USP_VARIANT_ANTISYMMETRIC = 1,
  USP_VARIANT_FLUX_DIFFUSION = 2
} usp_variant_kind;

typedef struct usp_variant usp_variant;

usp_status usp_variant_create(const usp_grid* grid, int32_t kind, const double* params,
                              const void* V, double alpha, void* cuda_stream,
                              usp_variant** out);

/* Algorithm 1 on (y, x): device pointers, K planes each; arguments and
 * results as usp_solve (refinements and stagnated are always 0). */
usp_status usp_variant_solve(usp_variant* s, const void* y, void* x, int32_t use_x0,
                             double tol, int32_t maxit, double ref_norm, usp_result* out);

/* Schedule of the variant's iterations (no counterpart in the paper): 0
 * automatic -- square 2-D grids n x n, n in {32, 64, 128}, keep the K
 * component fields of the problem in the shared memory of one thread-block
 * cluster and run a whole solve per launch, other grids use the passes; 1
 * the passes (pointwise kernels and the line / strided-axis transforms of
 * every component plane); 3 the on-chip kernel (USP_ERR_UNSUPPORTED_SIZE
 * where it does not apply).  Errors: USP_ERR_INVALID_ARG for other values. */
usp_status usp_variant_set_schedule(usp_variant* s, int32_t schedule);

/* Residual history of the last solve (as usp_residual_history). */
usp_status usp_variant_history(const usp_variant* s, double* host_out, int32_t capacity,
                               int32_t* n_out);

void usp_variant_destroy(usp_variant* s);

/* Host canonical forms (FP64 in, float32/complex64 out):
 * antisymmetrised Helmholtz laplacian psi + k^2 psi = -S (adjoint source
 *   S_adj, NULL for none): kbar2, rho = smallest circle of the values k^2,
 *   c = rho / norm_v (real), v = (k^2 - kbar2)/c (v_out: n complex64),
 *   l = (-|p|^2 + kbar2)/c (params_out: 4 doubles), y = [S_adj/c; -S/c]
 *   (y_out: 2 n complex64), c_out: 1 double.  k2, S, S_adj: n complex128.
 * flux-form diffusion -div(D grad u) + eta u = S: etabar, Dinvbar, r_eta,
 *   r_D = midpoints and half-ranges of eta and 1/D; c_u = r_eta/norm_v,
 *   c_J = r_D/norm_v (a zero range takes the other's); V_out: 2 n float32
 *   ((eta - etabar)/c_u, then (1/D - Dinvbar)/c_J); params_out: (etabar/c_u
 *   + 1, Dinvbar/c_J + 1, 1/sqrt(c_u c_J)); y_out: (1 + ndim) n complex64,
 *   [S/sqrt(c_u); 0]; scales_out: (c_u, c_J).  eta, D, S: n doubles
 *   (eta >= 0, D > 0); u = x[0] / sqrt(c_u). */
usp_status usp_canon_antisymmetric(const double* k2, const double* S, const double* S_adj,
                                   int64_t n, double norm_v, float* v_out, float* y_out,
                                   double* params_out, double* c_out);
usp_status usp_canon_flux_diffusion(const double* eta, const double* D, const double* S,
                                    int64_t n, int32_t ndim, double norm_v, float* V_out,
                                    float* y_out, double* params_out, double* scales_out);

/* ---- learned initial estimate (no counterpart in the paper) -------------
 *
 * Algorithm 1 starts from any x0 (Sec. 2.1; the paper's examples start at
 * 0).  This network -- a Fourier neural operator (Li et al. 2020) -- maps a
 * description of the medium and source to an estimate of the field, which a
 * solve then takes as x0 (use_x0 = 1, ref_norm <= 0: the stopping test keeps
 * the alpha-free denominator ||B (L+I)^-1 y||, so the answer is the
 * iteration's own).  Definition, per sample of c_in x h x w real inputs a:
 *   v_0 = P a + p (per pixel);  z_l = W_l v_l + b_l + K_l v_l;
 *   v_{l+1} = gelu(z_l) (l < layers - 1), v_layers = z_{layers-1};
 *   K_l v = Re F^-1[S^T R_l S F v] (F the unnormalised 2-D DFT, S keeps the
 *   modes x modes lowest frequencies: index k in [0, modes/2) or
 *   [n - modes/2, n) per axis; R_l a complex width x width matrix per mode);
 *   estimate = (Q v_layers + q)[0] + i (Q v_layers + q)[1];
 *   gelu(x) = x (1 + erf(x / sqrt 2)) / 2;
 *   loss = mean over the batch of ||estimate - x||^2 / ||x||^2.
 * Parameters (float32, this order): P [width][c_in], p [width]; per layer
 * W [width][width], b [width], R [width][width][modes][modes][re, im];
 * Q [2][width], q [2].  Training: the hand-derived backward pass and Adam
 * (beta 0.9, 0.999, eps 1e-8).  FP32 arithmetic, deterministic reductions.
 * Inputs a: device, batch x c_in x h x w float32; fields: device, batch x h
 * x w complex64. */
typedef struct {
  int32_t h, w;        /* image size, each in [8, 512]                       */
  int32_t c_in;        /* input channels, [1, 8]                             */
  int32_t width;       /* hidden channels, [1, 64]                           */
  int32_t layers;      /* spectral layers, [1, 8]                            */
  int32_t modes;       /* retained modes per axis, power of two in [2, 32]   */
  int32_t max_batch;   /* largest batch a call may pass                      */
} usp_fno_config;

typedef struct usp_fno usp_fno;

/* Number of parameters of a configuration (-1 if it is invalid). */
int64_t usp_fno_param_count(const usp_fno_config* cfg);

/* Create a network with parameters drawn from `seed` (uniform, scaled by
 * 1/sqrt(fan-in); R by 1/width^2; biases 0) and its activation memory for
 * max_batch samples; cuda_stream as in usp_solver_create. */
usp_status usp_fno_create(const usp_fno_config* cfg, uint64_t seed, void* cuda_stream,
                          usp_fno** out);

/* Copy the parameters out / in (host arrays of usp_fno_param_count
 * floats); setting them also resets the Adam state. */
usp_status usp_fno_get_params(const usp_fno* f, float* host_out, int64_t n);
usp_status usp_fno_set_params(usp_fno* f, const float* host_in, int64_t n);

/* Field estimate for `batch` samples into x_out (device complex64). */
usp_status usp_fno_predict(usp_fno* f, const float* a, int32_t batch, void* x_out);

/* Loss against x_true (device complex64) and its gradient with respect to
 * every parameter (host array, or NULL), without an update. */
usp_status usp_fno_gradients(usp_fno* f, const float* a, const void* x_true,
                             int32_t batch, float* grad_host, double* loss_out);

/* One training step: forward, loss, backward, Adam update with step size
 * lr.  *loss_out (may be NULL) receives the loss before the update. */
usp_status usp_fno_train_step(usp_fno* f, const float* a, const void* x_true,
                              int32_t batch, double lr, double* loss_out);

/* Free a network (NULL is ignored). */
void usp_fno_destroy(usp_fno* f);

/* ---- measurement (no counterpart in the paper; used by the benchmark) -- */

/* Mean duration of each kernel of one iteration. */
typedef struct {
  char name[32];      /* pass name, e.g. "rows_inv_post"                     */
  int32_t launches;   /* launches timed                                      */
  double ms;          /* mean duration per launch, CUDA events on the
                         solver's stream, milliseconds                        */
  double bytes;       /* algorithmic HBM bytes one launch moves (each input
                         read once, each output written once)                 */
} usp_pass_time;

/* Run `iters` iterations of the solver's schedule on (y, x) -- device
 * pointers as in usp_solve; x is overwritten -- after one untimed
 * iteration, launching every kernel directly and back to back with a CUDA
 * event between consecutive kernels, and report per-kernel mean durations
 * (device time between the kernel's neighbours' events; the host's launch
 * latency is hidden behind the kernel before).  out: host array of
 * `capacity` entries; *n_out = number of kernels per iteration. */
usp_status usp_time_passes(usp_solver* s, const void* y, void* x, int32_t iters,
                           usp_pass_time* out, int32_t capacity, int32_t* n_out);

/* Autotuner: time one iteration of each pass variant the solver's grid
 * admits (pencil, fused, split or on-chip schedule; TMA-staged or plain-load passes) over
 * `iters` iterations on (y, x) (device pointers; x is overwritten), keep the
 * fastest, and size the iterations per CUDA-graph launch (chunk) to about
 * 0.2 ms of GPU work.  The choice is cached per (grid, batch count, real or
 * complex V) for the process: a later solver of the same shape takes it
 * without timing.  Sets the solver's options (plain and max_refinements are
 * kept) and copies them to *chosen if not NULL. */
usp_status usp_autotune(usp_solver* s, const void* y, void* x, int32_t iters,
                        usp_options* chosen);

/* Number of kernel launches this library has issued in this process (a
 * CUDA-graph launch counts each kernel node it runs). */
int64_t usp_kernel_launches(void);

/* Human-readable name of a status code (static string). */
const char* usp_status_string(usp_status st);

/* Description of the last error on the calling thread (static storage,
 * valid until the next failing call on this thread). */
const char* usp_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int32_t usp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* USP_H */
