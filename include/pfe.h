/*
 * pfe.h -- C ABI of a single-GPU (GB300, sm_103a) polynomial-filtered interior eigensolver
 * for mass-weighted atomistic Hessians, after Accaputo, Derlet & Arbenz, "Solving large-scale
 * interior eigenvalue problems to investigate the vibrational properties of the boson peak
 * regime in amorphous materials" (arXiv 1902.07041).
 *
 * Problem (Sec. 1, eqs. (1)-(3)): given the 3x3-block Hessian Delta of a stable atomic
 * configuration and the masses m_i, find every eigenpair (lambda, q) of
 *     H q = lambda q,   H_ij = Delta_ij / sqrt(m_i m_j),   lambda = omega^2,
 * with lambda in a closed interval [a, b], ||q|| = 1, together with the residual norms
 * (Alg. 3).  The method is the Chebyshev-filtered subspace iteration of Sec. 2.6
 * (Alg. 2 for p_m(H) X, Alg. 4 with Rayleigh-Ritz and locking).
 *
 * Conventions shared by every call:
 *  - Every call returns a pfe_status; none aborts.  On failure pfe_last_error(ctx) gives a
 *    one-line message (thread-unsafe per context: one host thread per context at a time).
 *  - Matrices are 3x3 block CSR ("BSR") over atoms: row_ptr[N+1] (int32, row_ptr[0] = 0),
 *    col_idx[nnzb] (int32, ascending within a row, each row holds its diagonal block),
 *    vals[9 * nnzb] (float64, each block row-major: vals[9p + 3r + s] = block_p(r, s)).
 *  - Dense multivectors at the boundary are column-major n x k with a leading dimension
 *    ld >= n, n = 3N, dof index 3i + r for atom i, Cartesian component r.
 *  - Pointers are host pointers unless a flag or the call's description says "device".
 *    Device pointers must come from the same CUDA device the context was created on.
 *  - The caller keeps ownership of every buffer it passes; the library copies what it keeps.
 *  - Streams: the context runs its work on the stream given at creation (NULL = the legacy
 *    default stream).  Calls that take their own stream run their kernels on it.
 */
#ifndef PFE_H
#define PFE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfe_ctx pfe_ctx;

typedef enum {
  PFE_OK = 0,
  PFE_E_ARG = 1,       /* invalid argument (NULL, size, index out of range, NaN/Inf input) */
  PFE_E_NOMEM = 2,     /* host or device allocation failed */
  PFE_E_CUDA = 3,      /* a CUDA / cuBLAS / cuSOLVER call failed; message names it */
  PFE_E_NOTSYM = 4,    /* Delta is not symmetric: block (i,j) != block (j,i)^T beyond 1e-12 max|Delta| */
  PFE_E_CAPACITY = 5,  /* caller buffer or subspace width too small; counts are still reported */
  PFE_E_NOCONV = 6,    /* iteration limit reached before every interval eigenpair converged */
  PFE_E_BREAKDOWN = 7, /* orthogonalisation broke down even after the shifted retry */
  PFE_E_BOUND = 8,     /* lambda_max bound was violated (a Ritz value exceeded it) */
  PFE_E_TIMEOUT = 9,   /* a bounded device-side wait gave up */
  PFE_E_STATE = 10     /* call out of order (e.g. eigenpairs requested before a solve) */
} pfe_status;

/* flags for pfe_create and pfe_get_eigenpairs */
#define PFE_DEVICE_PTRS 0x1u    /* array arguments are device pointers */
#define PFE_SKIP_SYM_CHECK 0x2u /* do not verify the symmetry of Delta */

/* element types of pfe_filter_apply's X and Y */
#define PFE_F64 0 /* float64 vectors, float64 arithmetic */
#define PFE_F32 1 /* float32 vectors, float32 arithmetic (mixed-precision filter) */

/* parameter keys for pfe_set_param / pfe_get_param (values are doubles) */
enum {
  PFE_P_DEGREE = 1,         /* filter degree m; 0 = choose by eq. (thresh) (default 0) */
  PFE_P_EPS_FRAC = 2,       /* margin eps as a fraction of eta - xi (default 0.25) */
  PFE_P_RATE = 3,           /* convergence rate r of eq. (thresh) (default sqrt(0.1) for the subspace
                               iteration, 0.1^(1/4) for block Lanczos, METHOD 1) */
  PFE_P_DAMPING = 4,        /* 0 none (default, best for subspace iteration in Sec. 4.1), 1 Jackson, 2 Lanczos sigma */
  PFE_P_WIDTH = 5,          /* subspace width q; 0 = max(WIDTH_FACTOR * count estimate, 1.1 * window count
                               estimate + 8, MIN_WIDTH), the window being [a - eps, b + eps] (default 0) */
  PFE_P_WIDTH_FACTOR = 6,   /* default 1.5 */
  PFE_P_TOL = 7,            /* residual tolerance ||H v - lambda v|| / lambda_max_est (default 1e-8) */
  PFE_P_PRECISION = 8,      /* filter precision: 0 FP64 (default); 1 mixed: each Ritz pair is filtered in
                               FP32 while its residual exceeds REFINE_TOL, in FP64 after; 2 mixed by defect
                               correction: as 1, but below REFINE_TOL the pair's filter is split exactly into
                               x p(theta) in FP64 plus a recurrence on its residual H x - theta x in FP32 (no
                               FP64 filter sweep); the dense steps and residuals are FP64 in every mode */
  PFE_P_MAX_ITERS = 9,      /* subspace-iteration limit (default 60) */
  PFE_P_SEED = 10,          /* seed of the random start block and estimator vectors (default 0) */
  PFE_P_LAMBDA_MAX = 11,    /* spectrum upper bound; 0 = estimate by Lanczos (default 0) */
  PFE_P_LAMBDA_MIN = 12,    /* spectrum lower bound (default 0: H is positive semidefinite) */
  PFE_P_COUNT_M = 13,       /* number of estimator vectors M (default 30) */
  PFE_P_COUNT_DEGREE = 14,  /* estimator degree (default 100) */
  PFE_P_LANCZOS_STEPS = 15, /* Lanczos steps of the lambda_max estimate (default 30) */
  PFE_P_COUNT_DAMPING = 16, /* damping of the estimator series (default 0: plain truncation) */
  PFE_P_MIN_WIDTH = 17,     /* lower bound on the automatic width (default 16) */
  PFE_P_REFINE_TOL = 18,    /* mixed mode: residual below which a pair's filter runs in FP64 (default 1e-4) */
  PFE_P_STEP_SHAPE_F64 = 19, /* PROCESS-WIDE: kernel shape of the FP64 filter step, -1 = autotuned (default),
                               0 warp per (atom, column chunk), 1 CTA per 8 atoms x chunk, 2 and 3: the
                               same with two 3x3 blocks in flight per iteration, 4: neighbour rows staged
                               in shared memory by cp.async four blocks ahead (16-byte lanes), 5 and 6:
                               0 and 1 compiled for five resident CTAs per SM; 7, 8, 9: the rank-1
                               form (PFE_P_RANK1) as 0, 5 and 2 (shape 0 when there is none); 10 (only when
                               set, never autotuned): FP32 on the rank-1 form, a CTA per 32 atoms x 32
                               columns with the rows of the tile's neighbourhood staged in shared memory
                               (as 7 in FP64); 11: the rank-1 form as 8 compiled for six resident CTAs per
                               SM */
  PFE_P_STEP_SHAPE_F32 = 20, /* PROCESS-WIDE: the same for the FP32 filter step */
  PFE_P_METHOD = 21,        /* 0: filtered subspace iteration (Alg. 4, default); 1: thick-restart block
                               Lanczos on the filter operator (Sec. 2.5, the paper's Krylov-Schur solver),
                               FP64 only */
  PFE_P_BLOCK = 22,         /* block size of METHOD 1 (default 64) */
  PFE_P_BASIS_FACTOR = 23,  /* METHOD 1: basis size = BASIS_FACTOR x the wanted count (default 2; >= 1.25) */
  PFE_P_BATCH_THREADS = 24, /* pfe_solve_batch, read from the first context: host threads that run the
                               samples' set-up and dense steps concurrently, each sample on its own
                               stream (0 = automatic: min(samples, hardware threads, 16); 1 = serial) */
  PFE_P_RANK1 = 25,         /* 1 (default): when every off-diagonal block of H is -k r r^T / sqrt(m_i m_j)
                               (a central-force network, eqs. (1)-(2)) the filter steps use that rank-1
                               form, 6 FMAs a block and column instead of 9; 0: always the full 3x3
                               blocks.  pfe_get_param returns whether the form is in use (it is checked
                               when the filter operator is first built) */
  PFE_P_FILTER = 26,        /* 0 (default): the piecewise quadratic filter of eq. (fct_f) (both methods);
                               1: the Dirac filter of eq. (cheby-delta.1), METHOD 1 only (Sec. 2.5: the
                               paper's production choice with BKS) */
  PFE_P_PHI = 27,           /* Dirac filter degree: the smallest k whose filter, centred so that
                               rho(xi) = rho(eta), has rho(xi) / rho(gamma) <= PHI (default 0.8; the phi
                               of Tables 1-3) */
  PFE_P_DIRAC_CUT = 28,     /* Dirac filter with METHOD 1: Ritz values of rho(Ht) >= DIRAC_CUT x rho(xi) are
                               wanted (default 0.9) */
  PFE_P_SLICE_TARGET = 29,  /* pfe_solve_sliced: eigenvalues per slice the automatic edges aim at (default 1000) */
  PFE_P_OVERLAP = 30,       /* PRECISION 1: 1 filters an iteration's FP32 and FP64 column groups concurrently,
                               the FP32 group on a second stream of the context; 0 (default): one after the
                               other on the context's stream */
  PFE_P_DEGREE_RULE = 31    /* subspace iteration with the automatic degree (DEGREE 0, RATE not set):
                               1 (default) raises the degree of eq. (thresh) at r = sqrt(0.1) to the one in
                               [m, 4m] that minimises a model of the solve's work once the width is known
                               (iterations from the filter's largest value outside the margin window over its
                               smallest value in [a, b], times the filter and dense work of one); 0 keeps the
                               degree of eq. (thresh).  pfe_get_filter reports the degree in use (after a
                               solve, the one the solve used) */
};

/* ---------------------------------------------------------------------------------------
 * Setup (Sec. 3, Alg. 3; eq. (2) for the mass weighting)
 * ------------------------------------------------------------------------------------- */

/* Helper: assemble Delta of a spring network as BSR (eq. (1)): for every bond e = (i, j),
 * i != j, with stiffness k[e] and unit vector rhat[3e..3e+2] (from i to j),
 *   Delta_ij = Delta_ji = -k r r^T,  Delta_ii = -sum_{j != i} Delta_ij.
 * Two-call pattern: with cap_nnzb < required (e.g. 0 and NULL outputs) it only stores the
 * number of blocks in *nnzb and returns PFE_E_CAPACITY.  Host pointers, host computation.
 * Duplicate bonds are summed.  Returns PFE_E_ARG for i == j or an index out of [0, N). */
pfe_status pfe_springs_to_bsr(int32_t n_atoms, int64_t nbonds, const int32_t *bi, const int32_t *bj,
                              const double *k, const double *rhat, int64_t cap_nnzb, int32_t *row_ptr,
                              int32_t *col_idx, double *vals, int64_t *nnzb);

/* Create a solver context for H = M^-1/2 Delta M^-1/2 (eq. (2)).
 *   n_atoms N >= 1; nnzb = row_ptr[N]; masses[N] > 0, or NULL when vals already hold H.
 *   flags: PFE_DEVICE_PTRS (inputs on the device), PFE_SKIP_SYM_CHECK.
 *   cuda_stream: a cudaStream_t (NULL = default stream) used for all of the context's work.
 * The structure is validated on the host (ranges, ascending columns, diagonal present,
 * finite values, symmetry unless skipped).  Inputs are copied; H is formed on the device. */
pfe_status pfe_create(pfe_ctx **out, int32_t n_atoms, int64_t nnzb, const int32_t *row_ptr,
                      const int32_t *col_idx, const double *vals, const double *masses, uint32_t flags,
                      void *cuda_stream);

/* Release every device and host resource of the context (NULL is allowed). */
void pfe_destroy(pfe_ctx *ctx);

/* One-line description of the last failure on this context ("" if none). */
const char *pfe_last_error(const pfe_ctx *ctx);

pfe_status pfe_set_param(pfe_ctx *ctx, int key, double value);
pfe_status pfe_get_param(const pfe_ctx *ctx, int key, double *value);

/* The closed target interval [a, b] in lambda = omega^2 units, 0 <= a < b (eq. (intro.33)). */
pfe_status pfe_set_interval(pfe_ctx *ctx, double a, double b);

/* Alg. 3, set-up steps: bound lambda_max by a few Lanczos steps (unless PFE_P_LAMBDA_MAX is set),
 * form the transform of eq. (transf.1), and estimate the number of eigenvalues in [a, b]
 * with the stochastic trace estimator of Sec. 2.4 (eq. (eigval_count_estimator)).
 * Either output pointer may be NULL.  Needs an interval for the count (else count = NaN). */
pfe_status pfe_estimate(pfe_ctx *ctx, double *lambda_max, double *count_est);

/* The filter the solver uses (Alg. 3; eqs. (fct_f), (thresh), App. A; with PFE_P_FILTER = 1 the
 * Dirac filter of eq. (cheby-delta.1)): degree in *m
 * and the damped Chebyshev coefficients g_j gamma_j, j = 0..m, in coeffs[0..m] (host; may be
 * NULL to query m only, cap = its length); c and d of eq. (transf.1).  Runs pfe_estimate's
 * lambda_max step first if needed.  PFE_E_CAPACITY if cap < m + 1 (m still stored). */
pfe_status pfe_get_filter(pfe_ctx *ctx, int32_t cap, int32_t *m, double *coeffs, double *c, double *d);

/* The same filter design without a context (host computation only; no GPU needed), on the
 * transformed interval [xi, eta] within [-1, 1]:
 *   kind 0: the piecewise quadratic filter of eq. (fct_f) with margin eps and rate r (eq. (thresh));
 *   kind 1: the Dirac filter of eq. (cheby-delta.1), centred so that rho(xi) = rho(eta), with phi;
 * damping 0 none, 1 Jackson, 2 Lanczos (Sec. 2.3).  degree 0: the automatic degree (smallest
 * qualifying, as the solver picks it), else that degree (at most 60000, PFE_E_ARG above).  *m_out receives the degree;
 * coeffs[0..m] (host, cap doubles; may be NULL to query m) the damped Chebyshev coefficients.
 * PFE_E_ARG for an invalid interval or parameter or when no degree <= 60000 qualifies;
 * PFE_E_CAPACITY if cap < m + 1 (m still stored). */
pfe_status pfe_design_filter(int kind, double xi, double eta, double eps, double r, double phi, int damping,
                             int32_t degree, int32_t cap, int32_t *m_out, double *coeffs);

/* Alg. 3, solve step: compute all eigenpairs with lambda in [a, b] by filtered subspace iteration
 * (Alg. 4 with Rayleigh-Ritz on H every iteration, CholQR2 orthonormalisation, locking), or with
 * PFE_P_METHOD = 1 by thick-restart block Lanczos on p(Ht) followed by Rayleigh-Ritz with H.
 * *n_found receives their number.  Results stay in the context.
 * PFE_E_CAPACITY: the subspace was too narrow to certify completeness (raise PFE_P_WIDTH);
 * PFE_E_NOCONV: the iteration limit was hit (partial results are kept). */
pfe_status pfe_solve(pfe_ctx *ctx, int32_t *n_found);

/* The same filtered subspace iteration one outer iteration at a time (Alg. 4: each pass of its
 * loop is one application of p(Ht) to the active block, CholQR2 against the locked vectors,
 * Rayleigh-Ritz with H, residuals and locking).  pfe_solve is exactly
 *     pfe_solve_begin; do pfe_solve_iterate until *done; pfe_solve_end.
 * pfe_solve_begin: the set-up of pfe_solve (lambda_max bound and filter design if not yet done,
 *   count estimate, width, buffers, random start block and its orthonormalisation).  METHOD 0
 *   only (PFE_E_ARG otherwise); PFE_E_STATE without an interval.
 * pfe_solve_iterate: one outer iteration; *done (may be NULL) becomes 1 once the termination test
 *   of pfe_solve holds or the iteration limit is reached, after which further calls do nothing.
 *   Returns when the iteration's device work has finished.  On an error the solve is over.
 * pfe_solve_end: the results, as pfe_solve returns them.  Called before *done, it ends the solve
 *   early: the eigenpairs locked so far are the results and the status is PFE_E_NOCONV.
 * pfe_solve_iterate and pfe_solve_end return PFE_E_STATE when no stepwise solve is in progress. */
pfe_status pfe_solve_begin(pfe_ctx *ctx);
pfe_status pfe_solve_iterate(pfe_ctx *ctx, int32_t *done);
pfe_status pfe_solve_end(pfe_ctx *ctx, int32_t *n_found);

/* Copy the results of the last pfe_solve: lambda[cap] ascending, vecs n x cap column-major
 * (ld = n, unit 2-norm, mass-weighted coordinates q of eq. (3)), resid[cap] = ||H v - lambda v||
 * (absolute).  Any output may be NULL.  flags: PFE_DEVICE_PTRS for device output buffers.
 * PFE_E_CAPACITY if cap < n_found (nothing copied).  Also reports iteration statistics via
 * pfe_get_param-style keys in pfe_get_stats. */
pfe_status pfe_get_eigenpairs(pfe_ctx *ctx, int32_t cap, double *lambda, double *vecs, double *resid,
                              uint32_t flags);

/* Statistics of the last solve: iterations, single-vector products with H (the paper's
 * MatVec count, Sec. 4.1), subspace width, degree, filter seconds, total seconds. */
typedef struct {
  int32_t iterations;
  int32_t width;
  int32_t degree;
  int32_t n_found;
  int64_t matvecs;
  double lambda_max;
  double count_estimate;
  double seconds_total;
  double seconds_filter;
  double seconds_orth;
  double seconds_rr;
  double max_residual;
  int32_t fp64_sweeps; /* iterations in which some columns used the FP64 filter */
  int32_t status;
  double window_estimate; /* estimated eigenvalue count of the margin window (automatic width only) */
  int64_t kernel_launches;     /* launches of this library's own kernels since the context was created
                                  (process-wide counter: exact when one context works at a time) */
  int64_t filter_launches;     /* launches of the fused filter-step kernel inside the iteration */
  int64_t filter_col_steps;    /* sum over those launches of their column counts (FP64 filter) */
  int64_t filter_col_steps_f32;/* the same for the FP32 filter */
  double seconds_filter_f32;   /* part of seconds_filter spent in FP32 filter sweeps */
  int64_t batch_replays;       /* pfe_solve_batch: replays of the captured batched-filter graph */
  int32_t restarts;            /* METHOD 1: thick restarts */
  int32_t basis;               /* METHOD 1: maximal basis size */
  int32_t filter_shape_f64;    /* kernel shape of the last FP64 filter step (PFE_P_STEP_SHAPE_F64 numbering;
                                  7-9: the rank-1 form), -1 if none ran */
  int32_t filter_shape_f32;    /* the same for the FP32 filter step */
  int32_t slices;              /* pfe_solve_sliced: number of slices (0 for the other solves) */
  int32_t active;              /* stepwise solve in progress: columns still iterating (0 otherwise) */
  int32_t locked;              /* stepwise solve in progress: converged pairs locked so far (0 otherwise) */
  int32_t cholqr_shifts;       /* Cholesky factorisations of CholQR2 that broke down and were repeated
                                  with the shift of the retry (numerically rank-deficient blocks) */
  int64_t filter_col_steps_forced; /* PRECISION 2: the part of filter_col_steps_f32 run by the step with
                                  the forcing term (it also reads the residual block) */
} pfe_stats;
/* Between pfe_solve_begin and pfe_solve_end the counters iterations, matvecs, width, degree,
 * active, locked and kernel_launches describe the solve in progress; the other fields are those of
 * the last finished solve. */
pfe_status pfe_get_stats(const pfe_ctx *ctx, pfe_stats *stats);

/* ---------------------------------------------------------------------------------------
 * The filter (Alg. 2, the operator of Sec. 3) and its adjoint
 * ------------------------------------------------------------------------------------- */

/* Y = p_m(Ht) X with Ht = (H - cI)/d (eq. (transf.1)) and p_m = sum_{j<=m} coeffs[j] T_j
 * (Alg. 2; coeffs on the host, m + 1 of them, or NULL for the solver's own filter, in
 * which case m is ignored).  X and Y are DEVICE pointers, column-major n x k with leading
 * dimensions ldx, ldy >= n, element type dtype (PFE_F64 or PFE_F32, the same for X and Y;
 * PFE_F32 runs the recurrence in FP32 arithmetic).  Y must not overlap X.  k may be 0 (no-op).  c, d come from the context
 * (PFE_P_LAMBDA_MAX / _MIN or the Lanczos estimate).  stream: cudaStream_t or NULL for the
 * context's stream.  Work buffers are allocated by the context and kept for reuse. */
pfe_status pfe_filter_apply(pfe_ctx *ctx, int32_t m, const double *coeffs, int32_t k, const void *X,
                            int64_t ldx, void *Y, int64_t ldy, int dtype, void *stream);

/* Adjoint of Y = p_m(Ht) X for L = <Ybar, Y> with c, d held fixed (FP64 only):
 *   Xbar = p_m(Ht)^T Ybar = p_m(Ht) Ybar,
 *   vals_bar[9 nnzb] = dL/dH for each stored entry of H (same layout as vals).
 * The recurrence is recomputed from about sqrt(m) stored checkpoints of (t_j, t_{j-1}).
 * All arrays are DEVICE pointers; X, Ybar, Xbar column-major n x k.  vals_bar is overwritten. */
pfe_status pfe_filter_adjoint(pfe_ctx *ctx, int32_t m, const double *coeffs, int32_t k, const double *X,
                              int64_t ldx, const double *Ybar, int64_t ldyb, double *Xbar, int64_t ldxb,
                              double *vals_bar, void *stream);

/* Chain rule from vals_bar = dL/dH (per stored entry, as returned by pfe_filter_adjoint) to the
 * spring constants and masses of the network that pfe_springs_to_bsr assembled (eq. (2)):
 *   k_bar[e] = dL/dk_e,  m_bar[i] = dL/dm_i.
 * DEVICE pointers: bi, bj (int32), rhat (3 per bond), vals_bar, k_bar (nbonds), m_bar (N).
 * Needs a context created with masses. */
pfe_status pfe_chain_springs(pfe_ctx *ctx, int64_t nbonds, const int32_t *bi, const int32_t *bj,
                             const double *rhat, const double *vals_bar, double *k_bar, double *m_bar,
                             void *stream);

/* The filter of pfe_filter_apply (FP64) without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library allocate device
 * memory while they run -- applications whose device memory is already owned by another allocator
 * (a framework's caching allocator, or a pool sized at start-up), and loops that cannot afford the
 * implicit device synchronisation cudaMalloc and cudaFree may cause.
 * Its work buffers live in one fixed device array of 4 Mi doubles (32 MiB) inside the library:
 * every GPU that loads the library holds it until the process exits.  It needs
 * 4 * n * round_up(k, 4) doubles; larger problems get PFE_E_CAPACITY and nothing runs.
 * All calls share the array and it keeps the last call's contents; calls that overlap on the GPU
 * (other streams or host threads) race on it, so the caller serialises them.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.
 * Preconditions: the context already holds the FP64 filter operator for its current transform --
 * any earlier pfe_filter_apply, pfe_estimate or pfe_solve on it builds it (else PFE_E_STATE).
 * coeffs: host array of m + 1 coefficients (required); X, Y: device pointers, column-major n x k,
 * ld >= n, float64; stream as in pfe_filter_apply.  Given a stream other than the context's, the
 * call first waits on the host for the context's stream, where the filter operator was built.
 * It runs the kernel shape that pfe_filter_apply tuned for this column count (shape 0 before any
 * tuning), and does not time shapes itself. */
pfe_status pfe_filter_apply_noalloc(pfe_ctx *ctx, int32_t m, const double *coeffs, int32_t k, const double *X,
                                    int64_t ldx, double *Y, int64_t ldy, void *stream);

/* ---------------------------------------------------------------------------------------
 * Machine measurement (no counterpart in the paper)
 * ------------------------------------------------------------------------------------- */

/* The FP64 throughput this GPU sustains, the ceiling of every FP64 step of the method (the filter
 * step on GB300 is bound by the FP64 pipe).  Launches, on `stream` (a cudaStream_t, NULL = the
 * legacy default stream), kernels in which every thread advances 8 or 16 independent chains `iters`
 * times, with 4 or 8 CTAs of 256 threads per SM, either FMAs only or FMAs alternating with multiplies
 * (the mix of the filter step); for each shape the first launch warms up and the next `reps` are
 * timed with CUDA events on that stream.  *tflops receives the best rate, counting 2 flops per FP64
 * instruction (the convention of the filter step's flop count).  `sink` is one device double the kernels write only if a chain ends at a value
 * it cannot reach (it keeps the chains from being optimised away).  PFE_E_ARG for iters < 1,
 * reps < 1, NULL sink or tflops. */
pfe_status pfe_probe_fp64_fma(int32_t iters, int32_t reps, void *stream, double *sink, double *tflops);

/* ---------------------------------------------------------------------------------------
 * Batched solves of independent samples (the realisations H_1 .. H_8 of Sec. 4.2)
 * ------------------------------------------------------------------------------------- */

/* Solve every context's interval problem; n_found[s] per sample.  Each context must have its
 * interval set; all must live on one device.  The iterations of all samples advance in lockstep:
 * the filter of every FP64 sample runs as one persistent kernel per Chebyshev step over all
 * samples' work, captured once in a CUDA graph and replayed per iteration (its column tile and
 * grid size chosen by timing the candidates on the first call); the dense steps run per sample,
 * the samples' dense steps concurrently from PFE_P_BATCH_THREADS host threads.  When every context
 * selects PFE_P_METHOD = 1 the samples' block Lanczos solves run whole, concurrently from those
 * threads, each on its own stream, largest samples first; a finished sample's work buffers pass to
 * the next sample its thread solves (its eigenvectors stay), so only the solves in flight hold them
 * and none is freed while others run, and a sample that ran out of device memory beside the others
 * is solved again afterwards, alone.  All contexts of a batch select the same method (PFE_E_ARG otherwise).
 * In the stats of every sample seconds_filter is the batch's shared filter time.  In the lockstep
 * subspace iteration too, a sample that ran out of device memory beside the others is solved again
 * after the batch, alone (its stats are then its own solve's), and every sample releases its work
 * buffers when the batch ends (its eigenvectors stay).
 * Returns the first failing status (the other samples still run). */
pfe_status pfe_solve_batch(pfe_ctx **ctxs, int32_t nsamples, int32_t *n_found);

/* ---------------------------------------------------------------------------------------
 * Spectrum slicing (Sec. 2.6 and Sec. 5: split [a, b] into sub-intervals of a reasonable
 * eigenvalue count, e.g. for memory; Sec. 4.3 computes one interval as five)
 * ------------------------------------------------------------------------------------- */

/* All eigenpairs in the context's interval [a, b], computed slice by slice with the selected method
 * and merged; results and statistics as for pfe_solve (the statistics summed over the slices).
 * nedges = 0 (edges NULL): automatic edges, about PFE_P_SLICE_TARGET eigenvalues per slice, placed by
 * the cumulative count of the stochastic density of states (Sec. 2.4's estimator with Chebyshev
 * moments of degree D, so every slice count comes from one set of moments); one slice means pfe_solve.
 * Otherwise edges[0..nedges-1] (host) are the interior edges, strictly increasing inside (a, b).
 * Each slice is solved on its interval widened by 1e-6 lambda_max at its interior edges; the pairs
 * that two neighbouring slices return within 2e-6 lambda_max of their shared edge are merged by a
 * Rayleigh-Ritz step with H on their joint span (a pair found twice counts once).  Device memory:
 * the eigenvectors of all slices (n x found, FP64) beside one slice's solver buffers. */
pfe_status pfe_solve_sliced(pfe_ctx *ctx, int32_t nedges, const double *edges, int32_t *n_found);

/* ---------------------------------------------------------------------------------------
 * Analysis of the computed modes (Sec. 4.4).  A mode q is read as N 3-vectors q_i, the three
 * dof rows of atom i; both calls work on the context's found eigenvectors, on the device, in the
 * order of pfe_get_eigenpairs.  PFE_E_STATE without solve results; PFE_E_CAPACITY if cap < n_found.
 * ------------------------------------------------------------------------------------- */

/* Participation ratio of eq. (PR_def), normalised by the atom count so that a mode spread evenly
 * over all atoms gives 1, a single-atom mode 1/N and a plane wave 2/3:
 *     pr[s] = (sum_i |q_i|^2)^2 / (N sum_i |q_i|^4).
 * pr: host array of cap doubles. */
pfe_status pfe_participation_ratio(pfe_ctx *ctx, int32_t cap, double *pr);

/* Plane-wave content of each mode for nk wave vectors (the identification of sound modes by
 * wave vector k = 2 pi (m, n, l) / L and polarisation in Sec. 4.4).  With
 * A_d = sum_i q_{i,d} exp(i k . r_i) (d = x, y, z), k^ = k / |k|:
 *     out[2 (s nk + w)]     = (2/N) |k^ . A|^2 / |q|^2            (longitudinal)
 *     out[2 (s nk + w) + 1] = (2/N) (|A|^2 - |k^ . A|^2) / |q|^2  (transverse, both polarisations)
 * i.e. the weight of q on the plane waves sqrt(2/N) zeta sin(k . r_i), sqrt(2/N) zeta cos(k . r_i);
 * a plane wave of an allowed k gives 1 in its polarisation.  pos: host, 3N atom positions in the
 * atom order of H (any length unit); kvec: host, 3 nk components in the inverse unit, each nonzero
 * (PFE_E_ARG otherwise); out: host, 2 cap nk doubles. */
pfe_status pfe_plane_wave_content(pfe_ctx *ctx, const double *pos, int32_t nk, const double *kvec, int32_t cap,
                                  double *out);

#ifdef __cplusplus
}
#endif
#endif /* PFE_H */
