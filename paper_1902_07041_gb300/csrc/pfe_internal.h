// Internal declarations of the GB300 polynomial-filtered eigensolver library (libpfe).
// Host control (solver.cu), kernels (bsr_kernels.cu, vec_kernels.cu) and host math
// (filter_host.cu) meet here.  Nothing in this directory is shared with the CPU oracle.
#pragma once

#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pfe.h"

namespace pfe {

// Number of kernels this library has launched (all of its own kernels; cuBLAS/cuSOLVER excluded).
int64_t launch_count();
void count_launch();
void count_launches(int64_t n);  // launches replayed inside a CUDA graph
// Prefix of every kernel launch statement in this library: counts it, then launches.
#define PFE_LAUNCH ::pfe::count_launch(),

// --------------------------------------------------------------------------------------
// Device buffers
// --------------------------------------------------------------------------------------
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  template <typename T>
  T *as() const { return static_cast<T *>(p); }
};
cudaError_t dbuf_reserve(DBuf &b, size_t bytes);  // grow-only, contents not preserved
void dbuf_free(DBuf &b);

// --------------------------------------------------------------------------------------
// BSR matrix on the device (3x3 blocks, row-major inside a block)
// --------------------------------------------------------------------------------------
template <typename T>
struct Bsr {
  int32_t n_atoms = 0;
  const int32_t *rp = nullptr;
  const int32_t *ci = nullptr;
  const T *vals = nullptr;
  // Optional rank-1 form of the same operator (central-force networks): every off-diagonal block
  // is -u u^T.  rp1/ci1: the pattern without the diagonal blocks; u: 3 values per off-diagonal
  // block; dg: the symmetric diagonal block of each atom as (xx, xy, xz, yy, yz, zz).  Null when
  // the matrix does not have that form.
  const int32_t *rp1 = nullptr;
  const int32_t *ci1 = nullptr;
  const T *u = nullptr;
  const T *dg = nullptr;
  // tiles of 32 atoms for the shared-memory staged FP32 step (r1_tiled.cu): the union of each tile's
  // neighbourhoods, the slot of every off-diagonal block's column and of every atom in its tile
  const int32_t *tile_ptr = nullptr;
  const int32_t *tile_atoms = nullptr;
  const uint16_t *slot1 = nullptr;
  const uint16_t *self_slot = nullptr;
  int32_t tile_umax = 0;
};

// Step modes of the fused BSR kernel (row-major n x k multivectors with row stride ld):
//   SPMM : Z = alpha A X
//   FIRST: Z = alpha A X;              Y = g0 X + g1 Z
//   STEP : Z = alpha A X + beta W;     Y = Y + g1 Z        (W may alias Z; Y may be null)
//   STEP_ACC: as STEP with Y = Y + g0 X + g1 Z  (the term of X added one step late)
//   ADJ  : Z = alpha A X + beta W + g0 Y                   (Y read-only; W may alias Z)
enum StepMode { MODE_SPMM = 0, MODE_FIRST = 1, MODE_STEP = 2, MODE_ADJ = 3, MODE_STEP_ACC = 4 };

template <typename T>
void launch_bsr_step(const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z, T *Y, T alpha,
                     T beta, T g0, T g1, cudaStream_t s);
// kernel shape of the fused step (see bsr_kernels.cu): forced shape (-1 = autotuned) and the
// autotuner, which times every shape once per (type, columns per lane, chunk count)
void set_step_variant(int is_float, int variant);
int step_variant(int is_float);
// shape of the last filter-step launch (FIRST or STEP mode) of this type (process-wide; -1 before any), and a reset
int step_last_variant(int is_float);
void note_step_variant(int is_float, int variant);  // record the shape of a step launched outside launch_bsr_step
void reset_step_last_variant();
template <typename T>
void tune_step(const Bsr<T> &A, int32_t k, int64_t ld, const T *X, T *scratch, cudaStream_t s);
// the step on the rank-1 form (A.u, A.dg; shapes 0..2 of r1_kernels.cu)
template <typename T>
void dispatch_r1(int cpl, int variant, const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z,
                 T *Y, T alpha, T beta, T g0, T g1, cudaStream_t s);
// the FP32 step on the rank-1 form with each tile's neighbour rows staged in shared memory (shape 10);
// F, fs non-null add the forcing term fs[c] F of the defect correction
bool r1_tiled_usable(const Bsr<float> &A);
void launch_r1_tiled(const Bsr<float> &A, int mode, int32_t k, int64_t ld, const float *X, const float *W, float *Z,
                     float *Y, const float *F, const float *fs, float alpha, float beta, float g0, float g1,
                     cudaStream_t s);
void build_r1_tiles(int32_t n_atoms, const std::vector<int32_t> &rp1, const std::vector<int32_t> &ci1,
                    std::vector<int32_t> &tile_ptr, std::vector<int32_t> &tile_atoms, std::vector<uint16_t> &slot1,
                    std::vector<uint16_t> &self_slot, int32_t *umax);
// true when the autotuner chose the staged shape for FP32 steps on k columns
bool step_prefers_tiled(int32_t k, int64_t ld);
// true when the autotuner chose the rank-1 FP32 step at six resident CTAs per SM (shape 11) for k columns
bool step_prefers_six_ctas(int32_t k, int64_t ld);
// rank-1 form of alpha (H - shift I); *bad (device) is set to 1 if an off-diagonal block is not -u u^T
void launch_build_r1(int32_t n_atoms, const int32_t *rp, const int32_t *ci, const double *H, double alpha, double shift,
                     int32_t *rp1, int32_t *ci1, double *u64, double *dg64, float *u32, float *dg32, int32_t *bad,
                     cudaStream_t s);

// a0: H = Delta / sqrt(m_i m_j) per block; also the row index of each block
void launch_mass_weight(int32_t n_atoms, const int32_t *rp, const int32_t *ci, const double *delta, const double *mass,
                        double *H, cudaStream_t s);
// Filter operator Hs = alpha (H - shift I), in FP64 and (optionally) FP32
void launch_filter_matrix(int32_t n_atoms, const int32_t *rp, const int32_t *ci, const double *H, double alpha,
                          double shift, double *out64, float *out32, cudaStream_t s);
// Chain rule dL/dH (per stored entry) -> dL/dk, dL/dm
void launch_chain_springs(int32_t n_atoms, const int32_t *rp, const int32_t *ci, const double *H, const double *mass,
                          int64_t nbonds, const int32_t *bi, const int32_t *bj, const double *rhat, const double *hbar,
                          double *kbar, double *mbar, cudaStream_t s);
// Adjoint outer products over one checkpoint segment:
// hbar[9p + 3r + s] += sum_q alpha_q sum_c A_q[3i + r, c] T_q[3j + s, c] over every stored block p = (i, j),
// A_q = A0 + q stride, T_q = T0 + q stride, alpha_0 = alpha0, alpha_q = alpha (q >= 1); ld even
void launch_outer_accum_seg(const Bsr<double> &pattern, int64_t nnzb, int32_t k, int64_t ld, int32_t nq, int64_t stride,
                            const double *A0, const double *T0, double alpha0, double alpha, double *hbar, cudaStream_t s);

// --------------------------------------------------------------------------------------
// Dense helpers (row-major n x k blocks with row stride ld unless stated)
// --------------------------------------------------------------------------------------
// Philox4x32-10 normals: element (row i, column col0 + c) of stream `stream`
template <typename T>
void launch_fill_normal(uint64_t seed, uint32_t stream_id, int64_t n, int32_t k, int32_t col0, T *X, int64_t ld,
                        cudaStream_t s);
// out[c] = sum_i X[i,c] * Y[i,c] (deterministic two-pass); work >= colreduce_work(n, k) doubles
size_t colreduce_work(int64_t n, int32_t k);
template <typename T>
void launch_col_dots(int64_t n, int32_t k, const T *X, int64_t ldx, const T *Y, int64_t ldy, double *out, double *work,
                     cudaStream_t s);
// out[c] = || W[:,c] - theta[c] X[:,c] ||^2
void launch_col_resid2(int64_t n, int32_t k, const double *W, const double *X, int64_t ld, const double *theta,
                       double *out, double *work, cudaStream_t s);
template <typename T>
void launch_scale_cols(int64_t n, int32_t k, T *X, int64_t ld, const double *scale, cudaStream_t s);
template <typename T>
void launch_axpby(int64_t n, int32_t k, T alpha, const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, cudaStream_t s);
template <typename Tin, typename Tout>
void launch_convert(int64_t n, int32_t k, const Tin *X, int64_t ldx, Tout *Y, int64_t ldy, cudaStream_t s);
// dst[:, t] = src[:, idx[t]] (idx on the device)
void launch_gather_cols(int64_t n, int32_t kdst, const double *src, int64_t lds, double *dst, int64_t ldd,
                        const int32_t *idx, cudaStream_t s);
// column-major (n x k, ldc) <-> row-major (n x k, ldr)
template <typename T>
void launch_colmajor_to_rowmajor(int64_t n, int32_t k, const T *C, int64_t ldc, T *R, int64_t ldr, cudaStream_t s);
template <typename T>
void launch_rowmajor_to_colmajor(int64_t n, int32_t k, const T *R, int64_t ldr, T *C, int64_t ldc, cudaStream_t s);
template <typename T>
void launch_zero(T *p, int64_t count, cudaStream_t s);
// *out = max |G - I| over a k x k matrix (device scalar)
void launch_max_dev_identity(int32_t k, const double *G, double *out, cudaStream_t s);

// Batched filter: one persistent launch per Chebyshev step over every sample's work items.
// One descriptor per sample (device-resident, refreshed before every graph replay).
struct BatchDesc {
  const int32_t *rp;
  const int32_t *ci;
  const double *vals;  // filter operator A = (2/d)(H - cI)
  // its rank-1 form when the sample has one (u null otherwise): pattern without diagonal blocks,
  // 3 values per off-diagonal block, the symmetric diagonal blocks as (xx, xy, xz, yy, yz, zz)
  const int32_t *rp1, *ci1;
  const double *u, *dg;
  const double *X;
  double *b0, *b1, *Y;
  const double *coef;  // m + 1 damped coefficients
  int64_t ld;
  int64_t item_begin;  // prefix of items over samples
  int32_t n_atoms, k, m, nchunk;
};
void launch_batch_step(int cpl, int blocks, const BatchDesc *desc, int32_t nsamp, const int64_t *total, int32_t step,
                       cudaStream_t s);

// Mixed-precision filter by defect correction (defect.cu).  Step with forcing, FP32:
//   Z = A X - W + fs[c] F;  MODE_STEP: Y += g1 Z (Y may be null);  MODE_STEP_ACC: Y += g0 X + g1 Z
void launch_defect_step(const Bsr<float> &A, int mode, int32_t k, int64_t ld, const float *X, const float *W, float *Z,
                        float *Y, const float *F, const float *fs, float g0, float g1, cudaStream_t s,
                        bool six_ctas = false);
// start of a block whose first kd of act columns are defect columns (Rt = (W - theta X) inv_d):
//   defect: X32 = 0, B = Rt, F = Rt, Y32 = g1 Rt;  plain: X32 = X, F = 0
void launch_defect_prep(int64_t n, int32_t act, int32_t kd, const double *X, const double *W, int64_t ld,
                        const double *theta, double inv_d, double g1, float *X32, float *B, float *F, float *Y32,
                        cudaStream_t s);
// Y = pth[c] X + Y32 over act columns
void launch_defect_combine(int64_t n, int32_t act, const double *X, int64_t ld, const double *pth, const float *Y32,
                           double *Y, cudaStream_t s);

// --------------------------------------------------------------------------------------
// FP64 tensor-core (DMMA) products
// --------------------------------------------------------------------------------------
// C (m x nn, column-major ldc) = alpha A^T B + beta C for tall row-major A (K x m), B (K x nn);
// with sym (m == nn and A^T B symmetric, e.g. A == B or B = H A) only the upper tile triangle is computed
// and mirrored.
// work >= gram_work(K, m, nn, sym) doubles.
int32_t gram_splits(int64_t K, int32_t m, int32_t nn, bool sym);
size_t gram_work(int64_t K, int32_t m, int32_t nn, bool sym);
void launch_gram(int64_t K, int32_t m, int32_t nn, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double alpha, double beta, double *C, int64_t ldc, bool sym, double *work, cudaStream_t s);
// C (M x N row-major, ldc) = alpha A (M x K row-major, lda) Bc (K x N column-major, ldb) + beta C
void launch_update(int64_t M, int32_t N, int32_t K, const double *A, int64_t lda, const double *Bc, int64_t ldb,
                   double alpha, double beta, double *C, int64_t ldc, cudaStream_t s,
                   bool upper = false);

// --------------------------------------------------------------------------------------
// Host math of the filter (App. A, Sec. 2.3, eq. (thresh)); independent of the oracle
// --------------------------------------------------------------------------------------
// gamma_0..gamma_m of the piecewise quadratic p of eq. (fct_f)
void pq_coefficients(double xi, double eta, double eps, int32_t m, std::vector<double> &gamma);
// gamma_0..gamma_m of the characteristic function of [xi, eta]
void chi_coefficients(double xi, double eta, int32_t m, std::vector<double> &gamma);
// damping factors g_0..g_m (0 none, 1 Jackson, 2 Lanczos sigma)
void damping_factors(int kind, int32_t m, std::vector<double> &g);
// value of sum c_j T_j(x)
double chebyshev_value(const std::vector<double> &c, int32_t m, double x);
// smallest degree satisfying eq. (thresh), or -1
int32_t choose_degree(double xi, double eta, double eps, double r, int kind, int32_t kmax);
// largest |p| outside the margin window over the smallest p inside [xi, eta] (sampled)
double filter_ratio(const std::vector<double> &c, int32_t m, double xi, double eta, double eps);
// degree in [m0, 4 m0] minimising log(tol) / log(filter_ratio(m)) x (m + dense_steps)
int32_t choose_degree_cost(double xi, double eta, double eps, int kind, int32_t m0, double tol, double dense_steps);
// Dirac filter of eq. (cheby-delta.1): damped coefficients for centre gamma; the centre with equal
// values at xi and eta; the smallest degree whose balanced filter has rho(xi) / rho(gamma) <= phi
void dirac_coefficients(double gamma, int32_t m, int kind, std::vector<double> &c);
double dirac_center(double xi, double eta, int32_t m, int kind);
int32_t choose_dirac_degree(double xi, double eta, double phi, int kind, int32_t kmax);
// largest eigenvalue of a symmetric tridiagonal matrix and the last entry of its unit eigenvector
void tridiag_top(const std::vector<double> &alpha, const std::vector<double> &beta, double *theta, double *last);

}  // namespace pfe

// --------------------------------------------------------------------------------------
// State of one filtered subspace iteration (kept in the context between stages)
// --------------------------------------------------------------------------------------
struct SolveState {
  bool fp32 = false, use64 = true, was64 = true, done = false, timed_filter = true, timed32 = false;
  bool active = false;  // a stepwise solve (pfe_solve_begin .. pfe_solve_end) is in progress
  // PRECISION 2: the hand-over group is filtered in FP32 by defect correction (defect.cu) instead of FP64
  bool defect = false;
  std::vector<double> theta_act;     // Ritz values of the active columns, in their current order
  std::vector<double> h_pth;         // p(theta_t) per active column (0 for plain FP32 columns)
  std::vector<float> h_fs;           // 2 T_j(theta_t) per step j and column (row-major m x ld)
  float *R32 = nullptr, *dfs = nullptr;
  double *dtheta = nullptr, *dpth = nullptr;
  int32_t q = 0, act = 0, nl = 0, it = 0, prev_count = -1, fp64_sweeps = 0;
  int32_t k64 = 0;  // mixed precision: the first k64 active columns use the FP64 filter
  int64_t ld = 0, matvecs = 0, f_launch = 0, f_cols64 = 0, f_cols32 = 0, f_cols_forced = 0;
  double t_start = 0, t_filter = 0, t_filter32 = 0, t_orth = 0, t_rr = 0, prev_worst = 1e300, window_est = -1.0;
  pfe_status result = PFE_E_NOCONV;
  double *X = nullptr, *Y = nullptr, *W = nullptr, *T0 = nullptr, *T1 = nullptr, *L = nullptr;
  double *A = nullptr, *evals = nullptr, *red = nullptr, *resid2 = nullptr;
  int32_t *idx = nullptr;
  int *info = nullptr;
  float *X32 = nullptr, *Y32 = nullptr, *B32a = nullptr, *B32b = nullptr;
  std::vector<double> lockLam, lockRes, hth, hr2;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev32[2] = {nullptr, nullptr};
};

// --------------------------------------------------------------------------------------
// The context
// --------------------------------------------------------------------------------------
struct pfe_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // mixed precision: the FP32 column group of an iteration runs on `side` while the FP64 group runs on
  // `stream` (fork and join by events); created by the first mixed-precision solve
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t solver = nullptr;
  int32_t N = 0;
  int64_t n = 0;
  int64_t nnzb = 0;
  bool has_mass = false;
  pfe::DBuf rp, ci, H, mass, Hs64, Hs32;
  double hs_c = 0, hs_d = 0;  // transform the filter matrices were built for
  bool hs_valid = false, hs32_valid = false;
  // rank-1 form of the filter operator (central-force networks; see r1_kernels.cu):
  // r1_state -1 = not checked, 0 = H has no such form, 1 = built (r1_32: the FP32 copy too)
  pfe::DBuf r1_rp, r1_ci, r1_u64, r1_dg64, r1_u32, r1_dg32, r1_flag;
  int r1_state = -1;
  bool r1_32 = false;
  pfe::DBuf t_ptr, t_atoms, t_slot1, t_self;  // tiles of the staged FP32 step (built with the FP32 form)
  int32_t t_umax = 0;

  // parameters
  int32_t p_degree = 0;
  double p_eps_frac = 0.25;
  double p_rate = 0.0;  // 0: the method's default (rate_of)
  // r of eq. (thresh): the set value, else sqrt(0.1) for the subspace iteration (the locking paragraph
  // after Alg. 4) and 0.1^(1/4) for block Lanczos (its best piecewise-quadratic choice in Tables 1-3)
  double rate_of() const { return p_rate > 0.0 ? p_rate : (p_method == 1 ? 0.5623413251903491 : 0.31622776601683794); }
  int p_damping = 0;
  int32_t p_width = 0;
  double p_width_factor = 1.5;
  double p_tol = 1e-8;
  int p_precision = 0;
  int32_t p_max_iters = 60;
  uint64_t p_seed = 0;
  double p_lambda_max = 0, p_lambda_min = 0;
  int32_t p_count_m = 30, p_count_degree = 100, p_lanczos_steps = 30;
  int p_count_damping = 0;
  int32_t p_min_width = 16;
  double p_refine_tol = 1e-4;
  int p_overlap = 0;
  int p_degree_rule = 1;
  int p_method = 0;
  int32_t p_block = 64;
  double p_basis_factor = 2.0;
  int32_t p_batch_threads = 0;
  int p_rank1 = 1;
  int p_filter = 0;
  double p_phi = 0.8, p_dirac_cut = 0.9;
  int32_t p_slice_target = 1000;

  // state
  bool has_interval = false;
  double a = 0, b = 0;
  bool has_lmax = false;
  double lmax = 0, theta_max = 0, lanczos_resid = 0;
  bool has_count = false;
  double count_est = 0;
  bool has_filter = false;
  int32_t m = 0;
  int32_t m_thresh = 0;  // the degree of eq. (thresh) before any raise by the cost model
  std::vector<double> coef;
  double tc = 0, td = 0, xi = 0, eta = 0, eps = 0;
  double dirac_gamma = 0, dirac_tau = 0;  // Dirac filter: centre and the (equal) value at xi and eta

  // results
  bool has_result = false;
  int32_t n_found = 0;
  int32_t shift_count = 0;  // shifted Cholesky factorisations since the current solve began
  pfe::DBuf L;          // locked vectors, row-major n x ldq
  int64_t ldq = 0;
  std::vector<int32_t> result_cols;  // columns of L in ascending eigenvalue order
  std::vector<double> result_lam, result_res;
  pfe_stats stats{};

  // workspaces
  pfe::DBuf w_X, w_Y, w_W, w_T0, w_T1, w_T2, w_small, w_small2, w_red, w_idx, w_cs_work, w_info, w_f32a, w_f32b,
      w_f32c, w_f32d, w_ckpt, w_rr, w_gram, w_bks[5], w_slice[2], w_f32e, w_defect, w_tau;
  int64_t launch_base = 0;  // process-wide launch counter when the context was created
  SolveState solve;
  pfe::DBuf dcoef;            // filter coefficients on the device (batched solves)
  int tuned_cpl = 0, tuned_blocks = 0;  // autotuned batched-filter shape of the last batch
  std::string err;
};

// the thick-restart block Lanczos solve (bks.cu); uses the pieces below from solver.cu
pfe_status bks_solve(pfe_ctx *ctx, int32_t *n_found);
namespace pfe {
pfe_status solver_ensure_filter(pfe_ctx *ctx);
pfe_status solver_ensure_hs(pfe_ctx *ctx, bool need32);
pfe_status solver_count(pfe_ctx *ctx);
pfe_status solver_window(pfe_ctx *ctx, double *out);
// *shifted (optional): a factorisation broke down and was shifted (the block was numerically rank deficient)
pfe_status solver_cholqr2(pfe_ctx *ctx, double *Y, double *tmp, int32_t k, int64_t ld, double **result,
                          bool *shifted = nullptr);
pfe_status solver_filter64(pfe_ctx *ctx, int32_t k, int64_t ld, const double *X, double *Y, double *b0, double *b1);
// Y = sum_j coef[j] T_j(Ht) X on row-major n x ld blocks with the FP64 filter operator (its rank-1 form
// when built), on stream s; tune = false runs the already tuned kernel shape without timing candidates
pfe_status solver_filter64_rows(pfe_ctx *ctx, const double *coef, int32_t m, int32_t k, int64_t ld, const double *X,
                                double *Y, double *b0, double *b1, cudaStream_t s, bool tune);
double solver_now();
pfe_status solver_ensure_lmax(pfe_ctx *ctx);
Bsr<double> solver_bsr_H(const pfe_ctx *ctx);     // H
Bsr<double> solver_bsr_Hs64(const pfe_ctx *ctx);  // the filter operator A = (2/d)(H - cI)
}  // namespace pfe

// status helpers used across the host sources
pfe_status pfe_fail(pfe_ctx *ctx, pfe_status st, const std::string &msg);
#define PFE_CUDA_TRY(ctx, call)                                                                          \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return pfe_fail((ctx), PFE_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define PFE_BLAS_TRY(ctx, call)                                                                      \
  do {                                                                                               \
    cublasStatus_t e_ = (call);                                                                      \
    if (e_ != CUBLAS_STATUS_SUCCESS) return pfe_fail((ctx), PFE_E_CUDA, std::string(#call) + " failed (cublas " + std::to_string((int)e_) + ")"); \
  } while (0)
#define PFE_SOLVER_TRY(ctx, call)                                                                      \
  do {                                                                                                 \
    cusolverStatus_t e_ = (call);                                                                      \
    if (e_ != CUSOLVER_STATUS_SUCCESS) return pfe_fail((ctx), PFE_E_CUDA, std::string(#call) + " failed (cusolver " + std::to_string((int)e_) + ")"); \
  } while (0)
#define PFE_TRY(call)                    \
  do {                                   \
    pfe_status st_ = (call);             \
    if (st_ != PFE_OK) return st_;       \
  } while (0)
