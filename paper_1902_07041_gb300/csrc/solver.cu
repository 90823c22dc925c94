// The C ABI of libpfe and the host control of the filtered subspace iteration.
//
// Path of pfe_solve (Sec. 2.6, Alg. 3, Alg. 4 with Rayleigh-Ritz each iteration and locking):
//   Lanczos bound on lambda_max -> transform (eq. (transf.1)) -> coefficients and degree
//   (App. A, eq. (thresh)) -> eigenvalue-count estimate (Sec. 2.4) -> random start block ->
//   loop { Y = p_m(Ht) X (fused BSR kernel, m launches) ; Y -= L L^T Y ; CholQR2(Y) ;
//          W = H X ; Rayleigh-Ritz ; residuals ; lock } .
// The only device-to-host traffic per iteration is the q Ritz values and residual norms.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "pfe_internal.h"

using namespace pfe;

pfe_status pfe_fail(pfe_ctx *ctx, pfe_status st, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return st;
}

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

template <typename T>
T *reserve(pfe_ctx *ctx, DBuf &b, size_t count, pfe_status *st) {
  cudaError_t e = dbuf_reserve(b, count * sizeof(T));
  if (e != cudaSuccess) {
    *st = pfe_fail(ctx, PFE_E_NOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                         " bytes failed: " + cudaGetErrorString(e));
    return nullptr;
  }
  *st = PFE_OK;
  return b.as<T>();
}

#define RESERVE(T, ptr, buf, count)                 \
  T *ptr = nullptr;                                 \
  {                                                 \
    pfe_status st__;                                \
    ptr = reserve<T>(ctx, (buf), (count), &st__);   \
    if (st__ != PFE_OK) return st__;                \
  }

Bsr<double> bsr_H(const pfe_ctx *ctx) { return Bsr<double>{ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->H.as<double>()}; }
// the filter operator A = (2/d)(H - cI); with its rank-1 form when that was built and is enabled
Bsr<double> bsr_Hs64(const pfe_ctx *ctx) {
  Bsr<double> A{ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->Hs64.as<double>()};
  if (ctx->p_rank1 && ctx->r1_state == 1) {
    A.rp1 = ctx->r1_rp.as<int32_t>();
    A.ci1 = ctx->r1_ci.as<int32_t>();
    A.u = ctx->r1_u64.as<double>();
    A.dg = ctx->r1_dg64.as<double>();
  }
  return A;
}
Bsr<float> bsr_Hs32(const pfe_ctx *ctx) {
  Bsr<float> A{ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->Hs32.as<float>()};
  if (ctx->p_rank1 && ctx->r1_state == 1 && ctx->r1_32) {
    A.rp1 = ctx->r1_rp.as<int32_t>();
    A.ci1 = ctx->r1_ci.as<int32_t>();
    A.u = ctx->r1_u32.as<float>();
    A.dg = ctx->r1_dg32.as<float>();
    if (ctx->t_umax > 0) {
      A.tile_ptr = ctx->t_ptr.as<int32_t>();
      A.tile_atoms = ctx->t_atoms.as<int32_t>();
      A.slot1 = ctx->t_slot1.as<uint16_t>();
      A.self_slot = ctx->t_self.as<uint16_t>();
      A.tile_umax = ctx->t_umax;
    }
  }
  return A;
}

pfe_status check_launch(pfe_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return PFE_OK;
}

// ---------------------------------------------------------------- the filter driver (Alg. 2)
// Y = sum_j coef[j] T_j(Ht) X with A = (2/d)(H - cI) = 2 Ht:
//   t_1 = A t_0 / 2, t_{j+1} = A t_j - t_{j-1}; y accumulated in the same launch.
// X is read-only; b0, b1 are two scratch multivectors of the same shape.
// tune = false skips the shape autotuner (it synchronises the stream to time the candidates); the
// launches then take the shape already tuned for this type and column count, else shape 0.
template <typename T>
pfe_status run_filter(pfe_ctx *ctx, const Bsr<T> &A, const double *coef, int32_t m, int32_t k, int64_t ld, const T *X,
                      T *Y, T *b0, T *b1, cudaStream_t s, bool tune = true) {
  if (k <= 0) return PFE_OK;
  if (m == 0) {
    launch_axpby<T>(ctx->n, k, (T)coef[0], X, ld, T(0), Y, ld, s);
    return check_launch(ctx, "filter (degree 0)");
  }
  if (tune) tune_step<T>(A, k, ld, X, b1, s);  // b1 is free until the second step
  launch_bsr_step<T>(A, MODE_FIRST, k, ld, X, nullptr, b0, Y, T(0.5), T(0), (T)coef[0], (T)coef[1], s);
  const T *tprev = X;
  T *tcur = b0;
  // y is read and written every other step: an even step j adds g_j t_j (its input) and g_{j+1} t_{j+1}
  // (its output), an odd step adds nothing unless it is the last one (then g_m t_m)
  for (int32_t j = 1; j < m; ++j) {
    T *out = (tprev == X) ? b1 : const_cast<T *>(tprev);
    const bool even = (j % 2) == 0, last = j == m - 1;
    if (even)
      launch_bsr_step<T>(A, MODE_STEP_ACC, k, ld, tcur, tprev, out, Y, T(1), T(-1), (T)coef[j], (T)coef[j + 1], s);
    else
      launch_bsr_step<T>(A, MODE_STEP, k, ld, tcur, tprev, out, last ? Y : nullptr, T(1), T(-1), T(0),
                         (T)coef[j + 1], s);
    tprev = tcur;
    tcur = out;
  }
  return check_launch(ctx, "filter step");
}

// ---------------------------------------------------------------- set-up helpers
pfe_status ensure_lmax(pfe_ctx *ctx);

pfe_status lanczos_bound(pfe_ctx *ctx) {
  const int64_t n = ctx->n;
  const int32_t steps = (int32_t)std::min<int64_t>(std::max(ctx->p_lanczos_steps, 1), n);
  cudaStream_t s = ctx->stream;
  RESERVE(double, V, ctx->w_T0, (size_t)n * (steps + 1));
  RESERVE(double, w, ctx->w_T1, (size_t)n);
  RESERVE(double, h, ctx->w_small, (size_t)steps + 8);
  RESERVE(double, red, ctx->w_red, colreduce_work(n, 1) + 8);
  double *scal = h + steps + 1;  // one device scalar
  Bsr<double> A = bsr_H(ctx);
  launch_fill_normal<double>(ctx->p_seed, 1u, n, 1, 0, V, 1, s);
  launch_col_dots<double>(n, 1, V, 1, V, 1, scal, red, s);
  double nv = 0.0;
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&nv, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (!(nv > 0.0) || !std::isfinite(nv)) return pfe_fail(ctx, PFE_E_BREAKDOWN, "Lanczos start vector is zero");
  {
    std::vector<double> sc(1, 1.0 / std::sqrt(nv));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(scal, sc.data(), sizeof(double), cudaMemcpyHostToDevice, s));
    launch_scale_cols<double>(n, 1, V, 1, scal, s);
  }
  std::vector<double> al, be;
  const double one = 1.0, zero = 0.0, mone = -1.0;
  for (int32_t j = 0; j < steps; ++j) {
    double *vj = V + (int64_t)j * n;
    launch_bsr_step<double>(A, MODE_SPMM, 1, 1, vj, nullptr, w, nullptr, 1.0, 0.0, 0.0, 0.0, s);
    // full reorthogonalisation against v_0..v_j (two classical Gram-Schmidt passes); the first
    // pass also yields alpha_j = v_j^T w and removes alpha_j v_j + beta_{j-1} v_{j-1}
    double aj = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      PFE_BLAS_TRY(ctx, cublasDgemv(ctx->blas, CUBLAS_OP_T, (int)n, j + 1, &one, V, (int)n, w, 1, &zero, h, 1));
      if (pass == 0) {
        PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&aj, h + j, sizeof(double), cudaMemcpyDeviceToHost, s));
      }
      PFE_BLAS_TRY(ctx, cublasDgemv(ctx->blas, CUBLAS_OP_N, (int)n, j + 1, &mone, V, (int)n, h, 1, &one, w, 1));
    }
    launch_col_dots<double>(n, 1, w, 1, w, 1, scal, red, s);
    double bb = 0.0;
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&bb, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    al.push_back(aj);
    const double bj = std::sqrt(std::max(bb, 0.0));
    be.push_back(bj);
    if (!(bj > 1e-300) || j + 1 == steps) break;
    std::vector<double> sc(1, 1.0 / bj);
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(scal, sc.data(), sizeof(double), cudaMemcpyHostToDevice, s));
    launch_axpby<double>(n, 1, 1.0, w, 1, 0.0, V + (int64_t)(j + 1) * n, 1, s);
    launch_scale_cols<double>(n, 1, V + (int64_t)(j + 1) * n, 1, scal, s);
    PFE_TRY(check_launch(ctx, "Lanczos"));
  }
  double th = 0.0, last = 0.0;
  std::vector<double> offd(be.begin(), be.end() - 1);
  tridiag_top(al, offd, &th, &last);
  const double rb = std::fabs(be.back() * last);
  ctx->theta_max = th;
  ctx->lanczos_resid = rb;
  ctx->lmax = std::max(1.01 * th, th + rb);
  return PFE_OK;
}

void set_transform(pfe_ctx *ctx) {
  ctx->tc = 0.5 * (ctx->lmax + ctx->p_lambda_min);
  ctx->td = 0.5 * (ctx->lmax - ctx->p_lambda_min);
}

pfe_status ensure_lmax(pfe_ctx *ctx) {
  if (ctx->has_lmax) return PFE_OK;
  if (ctx->p_lambda_max > 0) {
    ctx->lmax = ctx->p_lambda_max;
    ctx->theta_max = ctx->lanczos_resid = 0;
  } else {
    PFE_TRY(lanczos_bound(ctx));
  }
  if (!(ctx->lmax > ctx->p_lambda_min)) return pfe_fail(ctx, PFE_E_ARG, "lambda_max must exceed lambda_min");
  set_transform(ctx);
  ctx->has_lmax = true;
  ctx->hs_valid = ctx->hs32_valid = false;
  return PFE_OK;
}

// Tiles of the shared-memory staged FP32 step (r1_tiled.cu), from the rank-1 pattern; once per context
// (the pattern does not change with the transform).  Without tiles the staged shape is never used.
pfe_status build_tiles(pfe_ctx *ctx) {
  const int64_t noff = ctx->nnzb - ctx->N;
  std::vector<int32_t> rp1((size_t)ctx->N + 1), ci1((size_t)noff);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(rp1.data(), ctx->r1_rp.p, sizeof(int32_t) * rp1.size(), cudaMemcpyDeviceToHost,
                                    ctx->stream));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(ci1.data(), ctx->r1_ci.p, sizeof(int32_t) * ci1.size(), cudaMemcpyDeviceToHost,
                                    ctx->stream));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<int32_t> tptr, tatoms;
  std::vector<uint16_t> slot1, self;
  int32_t umax = 0;
  build_r1_tiles(ctx->N, rp1, ci1, tptr, tatoms, slot1, self, &umax);
  if (umax <= 0) return PFE_OK;
  RESERVE(int32_t, dp, ctx->t_ptr, tptr.size());
  RESERVE(int32_t, da, ctx->t_atoms, tatoms.size());
  RESERVE(uint16_t, ds, ctx->t_slot1, std::max<size_t>(slot1.size(), 1));
  RESERVE(uint16_t, dself, ctx->t_self, self.size());
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(dp, tptr.data(), sizeof(int32_t) * tptr.size(), cudaMemcpyHostToDevice, ctx->stream));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(da, tatoms.data(), sizeof(int32_t) * tatoms.size(), cudaMemcpyHostToDevice,
                                    ctx->stream));
  if (!slot1.empty())
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(ds, slot1.data(), sizeof(uint16_t) * slot1.size(), cudaMemcpyHostToDevice,
                                      ctx->stream));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(dself, self.data(), sizeof(uint16_t) * self.size(), cudaMemcpyHostToDevice,
                                    ctx->stream));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // the host vectors must outlive the copies
  ctx->t_umax = umax;
  return PFE_OK;
}

pfe_status ensure_hs(pfe_ctx *ctx, bool need32) {
  PFE_TRY(ensure_lmax(ctx));
  const bool same = ctx->hs_c == ctx->tc && ctx->hs_d == ctx->td;
  if (same && ctx->hs_valid && (!need32 || ctx->hs32_valid)) return PFE_OK;
  RESERVE(double, h64, ctx->Hs64, (size_t)9 * ctx->nnzb);
  float *h32 = nullptr;
  if (need32) {
    RESERVE(float, p32, ctx->Hs32, (size_t)9 * ctx->nnzb);
    h32 = p32;
  }
  launch_filter_matrix(ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->H.as<double>(), 2.0 / ctx->td, ctx->tc,
                       h64, h32, ctx->stream);
  PFE_TRY(check_launch(ctx, "filter matrix"));
  if (ctx->p_rank1 && ctx->r1_state != 0 && ctx->nnzb > ctx->N) {
    const int64_t noff = ctx->nnzb - ctx->N;
    RESERVE(int32_t, rp1, ctx->r1_rp, (size_t)ctx->N + 1);
    RESERVE(int32_t, ci1, ctx->r1_ci, (size_t)noff);
    RESERVE(double, u64, ctx->r1_u64, 3 * (size_t)noff);
    RESERVE(double, dg64, ctx->r1_dg64, 6 * (size_t)ctx->N);
    float *u32 = nullptr, *dg32 = nullptr;
    const bool with32 = need32 || (same && ctx->hs32_valid);  // the FP32 operator in use after this call
    if (with32) {
      RESERVE(float, pu, ctx->r1_u32, 3 * (size_t)noff);
      RESERVE(float, pd, ctx->r1_dg32, 6 * (size_t)ctx->N);
      u32 = pu;
      dg32 = pd;
    }
    RESERVE(int32_t, flag, ctx->r1_flag, 1);
    PFE_CUDA_TRY(ctx, cudaMemsetAsync(flag, 0, sizeof(int32_t), ctx->stream));
    launch_build_r1(ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->H.as<double>(), 2.0 / ctx->td, ctx->tc,
                    rp1, ci1, u64, dg64, u32, dg32, flag, ctx->stream);
    PFE_TRY(check_launch(ctx, "rank-1 filter operator"));
    int32_t hbad = 1;
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hbad, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->r1_state = hbad ? 0 : 1;
    ctx->r1_32 = with32;
    if (!hbad && with32 && ctx->t_umax == 0) PFE_TRY(build_tiles(ctx));
    if (hbad) {
      for (DBuf *b : {&ctx->r1_rp, &ctx->r1_ci, &ctx->r1_u64, &ctx->r1_dg64, &ctx->r1_u32, &ctx->r1_dg32})
        dbuf_free(*b);
    }
  }
  ctx->hs_c = ctx->tc;
  ctx->hs_d = ctx->td;
  ctx->hs_valid = true;
  ctx->hs32_valid = need32 || (same && ctx->hs32_valid);
  return PFE_OK;
}

// damped coefficients of the piecewise quadratic filter of degree m (App. A, Sec. 2.3) into the context
void set_pq_filter(pfe_ctx *ctx, int32_t m) {
  std::vector<double> gam, g;
  pq_coefficients(ctx->xi, ctx->eta, ctx->eps, m, gam);
  damping_factors(ctx->p_damping, m, g);
  ctx->coef.resize((size_t)m + 1);
  for (int32_t j = 0; j <= m; ++j) ctx->coef[j] = gam[j] * g[j];
  ctx->m = m;
}

pfe_status ensure_filter(pfe_ctx *ctx) {
  if (ctx->has_filter) return PFE_OK;
  if (!ctx->has_interval) return pfe_fail(ctx, PFE_E_STATE, "no interval set (pfe_set_interval)");
  PFE_TRY(ensure_lmax(ctx));
  ctx->xi = (ctx->a - ctx->tc) / ctx->td;
  ctx->eta = (ctx->b - ctx->tc) / ctx->td;
  ctx->eps = ctx->p_eps_frac * (ctx->eta - ctx->xi);
  int32_t m = ctx->p_degree;
  if (ctx->p_filter == 1) {  // the Dirac filter of eq. (cheby-delta.1), centred so that rho(xi) = rho(eta)
    if (m <= 0) {
      m = choose_dirac_degree(ctx->xi, ctx->eta, ctx->p_phi, ctx->p_damping, 60000);
      if (m < 0) return pfe_fail(ctx, PFE_E_ARG, "no Dirac filter degree <= 60000 meets PHI");
    }
    ctx->dirac_gamma = dirac_center(ctx->xi, ctx->eta, m, ctx->p_damping);
    dirac_coefficients(ctx->dirac_gamma, m, ctx->p_damping, ctx->coef);
    ctx->dirac_tau = std::min(chebyshev_value(ctx->coef, m, ctx->xi), chebyshev_value(ctx->coef, m, ctx->eta));
    ctx->m = m;
    ctx->has_filter = true;
    return PFE_OK;
  }
  if (m <= 0) {
    m = choose_degree(ctx->xi, ctx->eta, ctx->eps, ctx->rate_of(), ctx->p_damping, 60000);
    if (m < 0) return pfe_fail(ctx, PFE_E_ARG, "no filter degree <= 60000 meets the rate; widen eps or r");
  }
  ctx->m_thresh = m;
  set_pq_filter(ctx, m);
  ctx->has_filter = true;
  return PFE_OK;
}

// The subspace iteration's automatic degree (no DEGREE, no RATE set, DEGREE_RULE 1): raised from the
// degree of eq. (thresh) at r = sqrt(0.1) to the one that minimises a model of the solve's work once the
// width q is known.  One filter step costs F per column (flops of the rank-1 or full-block operator);
// the dense steps of an iteration (Gram matrices and block updates of CholQR2, Rayleigh-Ritz and the
// projection) about 5.5 n q^2 flops; FP32 filter steps (mixed precision) are memory bound and cost
// about a tenth of an FP64 step (a half with the per-pair FP64 hand-over of PRECISION 1).
pfe_status apply_degree_rule(pfe_ctx *ctx, int32_t q) {
  if (ctx->p_degree_rule != 1 || ctx->p_degree > 0 || ctx->p_rate > 0.0 || ctx->p_filter != 0) return PFE_OK;
  const double n = (double)ctx->n, N = (double)ctx->N, nnzb = (double)ctx->nnzb;
  const bool r1 = ctx->p_rank1 && ctx->r1_state == 1;
  const double F = r1 ? 12.0 * (nnzb - N) + 18.0 * N + 6.0 * n : 18.0 * nnzb + 6.0 * n;
  const double rel = ctx->p_precision == 0 ? 1.0 : (ctx->p_precision == 1 ? 0.5 : 0.1);
  const double dense_steps = 5.5 * n * (double)q / F / rel;
  const int32_t m = choose_degree_cost(ctx->xi, ctx->eta, ctx->eps, ctx->p_damping, ctx->m_thresh, ctx->p_tol, dense_steps);
  if (m != ctx->m) set_pq_filter(ctx, m);
  return PFE_OK;
}

// Stochastic trace estimate of the number of eigenvalues in [lo, hi] (Sec. 2.4):
// T_M = (n / M) sum_l v_l^T psi(Ht) v_l with normalised Philox-Gaussian v_l (stream 2).
pfe_status estimate_count(pfe_ctx *ctx, double lo, double hi, double *out) {
  PFE_TRY(ensure_hs(ctx, false));
  const int64_t n = ctx->n;
  const int32_t M = std::max(ctx->p_count_m, 1), deg = std::max(ctx->p_count_degree, 0);
  const int64_t ld = round_up(M, 2);
  cudaStream_t s = ctx->stream;
  RESERVE(double, V, ctx->w_X, (size_t)n * ld);
  RESERVE(double, Y, ctx->w_Y, (size_t)n * ld);
  RESERVE(double, b0, ctx->w_T0, (size_t)n * ld);
  RESERVE(double, b1, ctx->w_T1, (size_t)n * ld);
  RESERVE(double, dots, ctx->w_small, (size_t)2 * M);
  RESERVE(double, red, ctx->w_red, colreduce_work(n, M));
  launch_zero<double>(V, n * ld, s);
  launch_fill_normal<double>(ctx->p_seed, 2u, n, M, 0, V, ld, s);
  launch_col_dots<double>(n, M, V, ld, V, ld, dots, red, s);
  std::vector<double> nrm(M);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(nrm.data(), dots, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  for (auto &v : nrm) v = 1.0 / std::sqrt(v);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(dots + M, nrm.data(), sizeof(double) * M, cudaMemcpyHostToDevice, s));
  launch_scale_cols<double>(n, M, V, ld, dots + M, s);
  const double xi = (lo - ctx->tc) / ctx->td, eta = (hi - ctx->tc) / ctx->td;
  std::vector<double> gam, g;
  chi_coefficients(xi, eta, deg, gam);
  damping_factors(ctx->p_count_damping, deg, g);
  for (int32_t j = 0; j <= deg; ++j) gam[j] *= g[j];
  PFE_TRY(run_filter<double>(ctx, bsr_Hs64(ctx), gam.data(), deg, M, ld, V, Y, b0, b1, s));
  launch_col_dots<double>(n, M, V, ld, Y, ld, dots, red, s);
  std::vector<double> vy(M);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(vy.data(), dots, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  double sum = 0.0;
  for (double v : vy) sum += v;
  *out = (double)n / (double)M * sum;
  return PFE_OK;
}

pfe_status count_estimate(pfe_ctx *ctx) {
  if (ctx->has_count) return PFE_OK;
  if (!ctx->has_interval) return pfe_fail(ctx, PFE_E_STATE, "no interval set (pfe_set_interval)");
  PFE_TRY(ensure_lmax(ctx));
  PFE_TRY(estimate_count(ctx, ctx->a, ctx->b, &ctx->count_est));
  ctx->has_count = true;
  return PFE_OK;
}

// The filter needs a subspace at least as wide as the number of eigenvalues in the margin
// window [xi - eps, eta + eps] (Sec. 2.6): estimate that count too.
pfe_status window_estimate(pfe_ctx *ctx, double *out) {
  PFE_TRY(ensure_filter(ctx));
  const double lo = ctx->tc + ctx->td * (ctx->xi - ctx->eps), hi = ctx->tc + ctx->td * (ctx->eta + ctx->eps);
  return estimate_count(ctx, std::max(lo, ctx->p_lambda_min), std::min(hi, ctx->lmax), out);
}

// ---------------------------------------------------------------- CholQR2 (+ shifted retry)
// G = Y^T Y by the DMMA Gram kernel (upper tiles, mirrored)
pfe_status gram_sym(pfe_ctx *ctx, const double *Y, int32_t k, int64_t ld, double *G) {
  RESERVE(double, gw, ctx->w_gram, gram_work(ctx->n, k, k, true));
  launch_gram(ctx->n, k, k, Y, ld, Y, ld, 1.0, 0.0, G, k, true, gw, ctx->stream);
  return check_launch(ctx, "Gram");
}

// R^T R = G (cuSOLVER potrf, upper) with the shifted retry of Fukaya et al. (2020): G + s I,
// s = 11 (n k + k (k + 1)) u trace(G); then Rinv = R^{-1} by a k x k triangular solve.
pfe_status chol_factor(pfe_ctx *ctx, double *G, double *Rinv, int32_t k, bool *shifted) {
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  RESERVE(int, info, ctx->w_info, 4);
  int lwork = 0;
  PFE_SOLVER_TRY(ctx, cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, k, G, k, &lwork));
  RESERVE(double, work, ctx->w_cs_work, (size_t)std::max(lwork, 1));
  std::vector<double> hG((size_t)k * k);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hG.data(), G, sizeof(double) * k * k, cudaMemcpyDeviceToHost, s));
  PFE_SOLVER_TRY(ctx, cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_UPPER, k, G, k, work, lwork, info));
  int hinfo = 0;
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  *shifted = false;
  if (hinfo != 0) {
    *shifted = true;
    ++ctx->shift_count;
    double tr = 0.0;
    for (int32_t i = 0; i < k; ++i) tr += hG[(size_t)i * k + i];
    const double sh = 11.0 * ((double)n * k + (double)k * (k + 1)) * 1.1102230246251565e-16 * tr;
    for (int32_t i = 0; i < k; ++i) hG[(size_t)i * k + i] += sh;
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(G, hG.data(), sizeof(double) * k * k, cudaMemcpyHostToDevice, s));
    PFE_SOLVER_TRY(ctx, cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_UPPER, k, G, k, work, lwork, info));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hinfo != 0) return pfe_fail(ctx, PFE_E_BREAKDOWN, "CholeskyQR broke down even with a shift");
  }
  std::vector<double> eye((size_t)k * k, 0.0);
  for (int32_t i = 0; i < k; ++i) eye[(size_t)i * k + i] = 1.0;
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(Rinv, eye.data(), sizeof(double) * k * k, cudaMemcpyHostToDevice, s));
  const double one = 1.0;
  PFE_BLAS_TRY(ctx, cublasDtrsm(ctx->blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT,
                                k, k, &one, G, k, Rinv, k));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // eye must outlive its copy
  return PFE_OK;
}

// CholQR2 of Y into an orthonormal Q (Y is n x k, row-major, row stride ld), using tmp as the
// second buffer; *result points to whichever holds Q.  Pass 1: G = Y^T Y, Y R^{-1} -> tmp.
// Pass 2 only if the Gram matrix of tmp deviates from I by more than 1e-13 (max entry), and
// a third pass after a shifted factorisation.
// gram_out (optional): when the block after the first pass is already nearly orthonormal (its Gram
// matrix G1 within 1e-3 of I, no shift), the second pass is left to the caller, which folds it into a
// generalized Rayleigh-Ritz problem (X1^T H X1) c = theta G1 c: *gram_out then points to G1 (device,
// k x k, valid until the next CholQR2) and *result to the once-orthonormalised block.  Otherwise
// *gram_out is null and *result is orthonormal.
pfe_status cholqr2(pfe_ctx *ctx, double *Y, double *tmp, int32_t k, int64_t ld, double **result, bool *shifted_out = nullptr,
                   double **gram_out = nullptr) {
  *result = Y;
  if (shifted_out) *shifted_out = false;
  if (gram_out) *gram_out = nullptr;
  if (k <= 0) return PFE_OK;
  cudaStream_t s = ctx->stream;
  RESERVE(double, G, ctx->w_small, (size_t)2 * k * k + 8);
  double *Rinv = G + (size_t)k * k, *dev = G + 2 * (size_t)k * k;
  double *src = Y, *dst = tmp;
  bool any_shift = false;
  for (int pass = 0; pass < 3; ++pass) {
    if (pass == 2 && !any_shift) break;  // the third pass only follows a shifted factorisation
    PFE_TRY(gram_sym(ctx, src, k, ld, G));
    if (pass > 0) {
      launch_max_dev_identity(k, G, dev, s);
      double h = 1.0;
      PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&h, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
      PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
      if (h <= 1e-13 && !(any_shift && pass == 1)) break;
      if (gram_out && pass == 1 && !any_shift && h <= 1e-3) {
        *gram_out = G;
        break;
      }
    }
    bool shifted = false;
    PFE_TRY(chol_factor(ctx, G, Rinv, k, &shifted));
    any_shift = any_shift || shifted;
    launch_update(ctx->n, k, k, src, ld, Rinv, k, 1.0, 0.0, dst, ld, s, true);  // R^{-1} is upper triangular
    PFE_TRY(check_launch(ctx, "CholeskyQR update"));
    *result = dst;
    std::swap(src, dst);
  }
  if (shifted_out) *shifted_out = any_shift;
  return PFE_OK;
}

// Y <- Y - L (L^T Y): one classical Gram-Schmidt pass against the locked block (DMMA products).
// The locked vectors are converged eigenvectors and the active block was orthogonal to them before
// the filter, so the filtered block's component along them is small and one pass suffices.
pfe_status project_out(pfe_ctx *ctx, const double *L, int32_t nl, double *Y, int32_t k, int64_t ld) {
  if (nl <= 0 || k <= 0) return PFE_OK;
  const int64_t n = ctx->n;
  RESERVE(double, h, ctx->w_small2, (size_t)nl * k);
  RESERVE(double, gw, ctx->w_gram, gram_work(n, nl, k, false));
  launch_gram(n, nl, k, L, ld, Y, ld, 1.0, 0.0, h, nl, false, gw, ctx->stream);
  launch_update(n, k, nl, L, ld, h, nl, -1.0, 1.0, Y, ld, ctx->stream);
  return check_launch(ctx, "projection");
}

// ---------------------------------------------------------------- the solve, in stages
// solve_setup: filter design, width, buffers, random start block.  solve_filter: Y = p(Ht) X
// on the active columns.  solve_after_filter: project out the locked block, CholQR2,
// Rayleigh-Ritz, residuals, locking and the termination test.  solve_finish: results.
// pfe_solve runs them for one context; pfe_solve_batch interleaves many contexts and replaces
// solve_filter by one batched persistent launch per Chebyshev step.
pfe_status solve_setup(pfe_ctx *ctx) {
  SolveState &st = ctx->solve;
  if (ctx->p_filter != 0)
    return pfe_fail(ctx, PFE_E_ARG, "the subspace iteration uses the piecewise quadratic filter (FILTER 0); "
                                    "the Dirac filter is for the block Lanczos method (METHOD 1)");
  for (int e = 0; e < 4; ++e)
    if (st.ev[e]) cudaEventDestroy(st.ev[e]);
  for (int e = 0; e < 2; ++e)
    if (st.ev32[e]) cudaEventDestroy(st.ev32[e]);
  st = SolveState{};
  if (!ctx->has_interval) return pfe_fail(ctx, PFE_E_STATE, "no interval set (pfe_set_interval)");
  st.t_start = now_s();
  ctx->has_result = false;
  ctx->n_found = 0;
  ctx->stats = pfe_stats{};
  ctx->shift_count = 0;
  st.fp32 = ctx->p_precision >= 1;
  st.defect = ctx->p_precision == 2;
  PFE_TRY(ensure_filter(ctx));
  PFE_TRY(ensure_hs(ctx, st.fp32));
  int32_t q = ctx->p_width;
  if (q <= 0) {
    PFE_TRY(count_estimate(ctx));
    PFE_TRY(window_estimate(ctx, &st.window_est));
    const double qa = ctx->p_width_factor * std::max(ctx->count_est, 0.0);
    const double qw = 1.1 * std::max(st.window_est, 0.0) + 8.0;
    q = (int32_t)std::ceil(std::max(qa, qw));
    q = std::max(q, ctx->p_min_width);
  }
  q = (int32_t)std::min<int64_t>(q, ctx->n);
  PFE_TRY(apply_degree_rule(ctx, q));
  const int64_t n = ctx->n, ld = round_up(q, 4);
  st.q = q;
  st.ld = ld;
  ctx->ldq = ld;
  cudaStream_t s = ctx->stream;
  const size_t big = (size_t)n * ld;
  RESERVE(double, X, ctx->w_X, big);
  RESERVE(double, Y, ctx->w_Y, big);
  RESERVE(double, W, ctx->w_W, big);
  RESERVE(double, T0, ctx->w_T0, big);
  RESERVE(double, T1, ctx->w_T1, big);
  RESERVE(double, L, ctx->L, big);
  RESERVE(double, A, ctx->w_rr, (size_t)q * q + (size_t)q + 8);
  RESERVE(double, red, ctx->w_red, colreduce_work(n, q) + (size_t)q + 8);
  RESERVE(int32_t, idx, ctx->w_idx, (size_t)q + 8);
  RESERVE(int, info, ctx->w_info, 4);
  st.X = X; st.Y = Y; st.W = W; st.T0 = T0; st.T1 = T1; st.L = L;
  st.A = A;
  st.evals = A + (size_t)q * q;
  st.red = red;
  st.resid2 = red + colreduce_work(n, q);
  st.idx = idx;
  st.info = info;
  if (st.fp32 && !ctx->side) {
    PFE_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    PFE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    PFE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  }
  if (st.fp32) {
    RESERVE(float, x32, ctx->w_f32a, big);
    RESERVE(float, y32, ctx->w_f32b, big);
    RESERVE(float, a32, ctx->w_f32c, big);
    RESERVE(float, b32, ctx->w_f32d, big);
    st.X32 = x32; st.Y32 = y32; st.B32a = a32; st.B32b = b32;
    for (float *p : {x32, y32, a32, b32}) launch_zero<float>(p, (int64_t)big, s);
    if (st.defect) {
      RESERVE(float, r32, ctx->w_f32e, big);
      RESERVE(double, dd, ctx->w_defect, 2 * (size_t)ld + 8);
      RESERVE(float, tau, ctx->w_tau, (size_t)std::max(ctx->m, 1) * ld);
      launch_zero<float>(r32, (int64_t)big, s);
      st.R32 = r32;
      st.dtheta = dd;
      st.dpth = dd + ld;
      st.dfs = tau;
    }
  }
  for (double *p : {X, Y, W, T0, T1, L}) launch_zero<double>(p, (int64_t)big, s);
  for (int e = 0; e < 4; ++e)
    if (!st.ev[e]) PFE_CUDA_TRY(ctx, cudaEventCreate(&st.ev[e]));
  for (int e = 0; e < 2; ++e)
    if (!st.ev32[e]) PFE_CUDA_TRY(ctx, cudaEventCreate(&st.ev32[e]));
  // start block: stream 0 of the seeded Philox normals, columns scaled to unit norm.  It is not
  // orthonormalised: the first filter application maps it to p(Ht) X0, whose span is that of
  // p(Ht) X0 R^-1 for any invertible R, and the filtered block is orthonormalised (CholQR2) anyway.
  launch_fill_normal<double>(ctx->p_seed, 0u, n, q, 0, st.X, ld, s);
  PFE_TRY(check_launch(ctx, "start block"));
  {
    RESERVE(double, dots, ctx->w_small, 2 * (size_t)q + 8);
    launch_col_dots<double>(n, q, st.X, ld, st.X, ld, dots, st.red, s);
    std::vector<double> nrm((size_t)q);
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(nrm.data(), dots, sizeof(double) * q, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    for (double &v : nrm) v = v > 0.0 ? 1.0 / std::sqrt(v) : 1.0;
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(dots + q, nrm.data(), sizeof(double) * q, cudaMemcpyHostToDevice, s));
    launch_scale_cols<double>(n, q, st.X, ld, dots + q, s);
    PFE_TRY(check_launch(ctx, "start block scaling"));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // nrm must outlive its copy
  }
  st.act = q;
  st.use64 = !st.fp32;
  st.k64 = st.fp32 ? 0 : q;
  st.hth.resize(q);
  st.hr2.resize(q);
  st.it = 0;
  return PFE_OK;
}

// PRECISION 2: the first kd active columns (residual below the hand-over tolerance) are filtered by
// defect correction, the others by the plain FP32 recurrence, all in one FP32 launch per step:
//   prep (Rt = (W - X Theta)/d for the defect columns; X rounded for the plain ones), the first step of
//   the plain columns, steps 1 .. m-1 with the forcing 2 T_j(theta_t) Rt, then Y = X p(Theta_t) + Y32.
pfe_status solve_filter_defect(pfe_ctx *ctx, int32_t kd) {
  SolveState &st = ctx->solve;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n, ld = st.ld;
  const int32_t act = st.act, m = ctx->m, kp = act - kd;
  const std::vector<double> &g = ctx->coef;
  if (m < 1) {  // degree 0: y = g0 x
    launch_axpby<double>(n, act, g[0], st.X, ld, 0.0, st.Y, ld, s);
    return check_launch(ctx, "filter (degree 0)");
  }
  if ((int32_t)st.theta_act.size() < kd) return pfe_fail(ctx, PFE_E_STATE, "defect filter without Ritz values");
  // host: theta_t, the Chebyshev values T_j(theta_t) (three-term recurrence), p(theta_t)
  st.h_pth.assign((size_t)act, 0.0);
  st.h_fs.assign((size_t)m * ld, 0.f);
  for (int32_t c = 0; c < kd; ++c) {
    const double tt = (st.theta_act[c] - ctx->tc) / ctx->td;
    double tm = 1.0, tj = tt, p = g[0] + g[1] * tt;
    for (int32_t j = 1; j < m; ++j) {
      st.h_fs[(size_t)j * ld + c] = (float)(2.0 * tj);
      const double tn = 2.0 * tt * tj - tm;
      tm = tj;
      tj = tn;
      p += g[j + 1] * tj;
    }
    st.h_pth[c] = p;
  }
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(st.dtheta, st.theta_act.data(), sizeof(double) * kd, cudaMemcpyHostToDevice, s));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(st.dpth, st.h_pth.data(), sizeof(double) * act, cudaMemcpyHostToDevice, s));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(st.dfs, st.h_fs.data(), sizeof(float) * st.h_fs.size(), cudaMemcpyHostToDevice, s));
  cudaEventRecord(st.ev32[0], s);
  const Bsr<float> A = bsr_Hs32(ctx);
  launch_defect_prep(n, act, kd, st.X, st.W, ld, st.dtheta, 1.0 / ctx->td, g[1], st.X32, st.B32a, st.R32, st.Y32, s);
  tune_step<float>(A, act, ld, st.X32, st.B32b, s);  // B32b is free until step 1
  const bool tiled = step_prefers_tiled(act, ld) && r1_tiled_usable(A) && ld % 4 == 0;  // buffers 16-byte aligned
  const bool six = step_prefers_six_ctas(act, ld);
  if (kp > 0)  // t_1 = A t_0 / 2 and y = g0 t_0 + g1 t_1 for the plain columns
    launch_bsr_step<float>(A, MODE_FIRST, kp, ld, st.X32 + kd, nullptr, st.B32a + kd, st.Y32 + kd, 0.5f, 0.f,
                           (float)g[0], (float)g[1], s);
  const float *tprev = st.X32;
  float *tcur = st.B32a;
  for (int32_t j = 1; j < m; ++j) {
    float *out = (tprev == st.X32) ? st.B32b : const_cast<float *>(tprev);
    const bool even = (j % 2) == 0, last = j == m - 1;
    if (tiled)
      launch_r1_tiled(A, even ? MODE_STEP_ACC : MODE_STEP, act, ld, tcur, tprev, out, (even || last) ? st.Y32 : nullptr,
                      st.R32, st.dfs + (size_t)j * ld, 1.f, -1.f, (float)g[j], (float)g[j + 1], s);
    else
      launch_defect_step(A, even ? MODE_STEP_ACC : MODE_STEP, act, ld, tcur, tprev, out,
                         (even || last) ? st.Y32 : nullptr, st.R32, st.dfs + (size_t)j * ld, (float)g[j], (float)g[j + 1],
                         s, six);
    tprev = tcur;
    tcur = out;
  }
  launch_defect_combine(n, act, st.X, ld, st.dpth, st.Y32, st.Y, s);
  if (m > 1) note_step_variant(1, tiled ? 10 : (six ? 11 : 8));  // the forced steps: as shape 10, 11 or 8
  cudaEventRecord(st.ev32[1], s);
  st.timed32 = true;
  st.was64 = false;
  st.f_launch += m;
  st.f_cols32 += (int64_t)act * m;
  st.f_cols_forced += (int64_t)act * (m - 1);
  st.matvecs += (int64_t)act * m;
  return check_launch(ctx, "defect-corrected filter");
}

// Y = p(Ht) X on the active columns (the single-context path).  In the mixed-precision mode the
// active block is ordered [FP64 columns | FP32 columns]: pairs whose residual is already below the
// hand-over tolerance are filtered in FP64, the others in FP32 (st.k64 columns in FP64).
pfe_status solve_filter(pfe_ctx *ctx) {
  SolveState &st = ctx->solve;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n, ld = st.ld;
  const int32_t m1 = std::max(ctx->m, 1);
  const int32_t k64 = st.fp32 ? std::min(st.k64, st.act) : st.act;
  const int32_t k32 = st.act - k64;
  st.was64 = k32 == 0;
  // Both groups present: the FP32 group (bound by memory latency and bandwidth) runs on the side
  // stream concurrently with the FP64 group (bound by the FP64 pipe).  They touch disjoint columns:
  // the FP64 group is a multiple of 4 columns, so its vector lanes end before column k64.
  if (st.defect && k64 > 0) return solve_filter_defect(ctx, k64);
  const bool split = k64 > 0 && k32 > 0 && ctx->p_overlap && ctx->side;
  cudaStream_t s32 = split ? ctx->side : s;
  if (split) {
    PFE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, s));
    PFE_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  }
  if (k32 > 0) {
    cudaEventRecord(st.ev32[0], s32);
    st.f_launch += m1;
    st.f_cols32 += (int64_t)k32 * m1;
    launch_convert<double, float>(n, k32, st.X + k64, ld, st.X32 + k64, ld, s32);
    PFE_TRY(run_filter<float>(ctx, bsr_Hs32(ctx), ctx->coef.data(), ctx->m, k32, ld, st.X32 + k64, st.Y32 + k64,
                              st.B32a + k64, st.B32b + k64, s32));
    launch_convert<float, double>(n, k32, st.Y32 + k64, ld, st.Y + k64, ld, s32);
    cudaEventRecord(st.ev32[1], s32);
    st.timed32 = true;
  }
  if (k64 > 0) {
    st.f_launch += m1;
    st.f_cols64 += (int64_t)k64 * m1;
    PFE_TRY(run_filter<double>(ctx, bsr_Hs64(ctx), ctx->coef.data(), ctx->m, k64, ld, st.X, st.Y, st.T0, st.T1, s));
    ++st.fp64_sweeps;
  }
  if (split) {
    PFE_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
    PFE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));
  }
  st.matvecs += (int64_t)st.act * ctx->m;
  return PFE_OK;
}

// Everything of one iteration after the filter; sets st.done when the solve has ended.
pfe_status solve_after_filter(pfe_ctx *ctx) {
  SolveState &st = ctx->solve;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n, ld = st.ld;
  const int32_t q = st.q;
  ++st.it;
  const int32_t act = st.act;
  cudaEventRecord(st.ev[1], s);
  // ---- orthonormalise against the locked vectors and within the block
  PFE_TRY(project_out(ctx, st.L, st.nl, st.Y, act, ld));
  double *G1 = nullptr;  // set: the block is once-orthonormalised, its Gram matrix G1 joins Rayleigh-Ritz
  {
    double *res = nullptr;
    PFE_TRY(cholqr2(ctx, st.Y, st.T0, act, ld, &res, nullptr, &G1));
    if (res != st.Y) std::swap(st.Y, st.T0);
  }
  std::swap(st.X, st.Y);
  cudaEventRecord(st.ev[2], s);
  // ---- Rayleigh-Ritz with H: W = H X, A = X^T W, A = Q Theta Q^T, X <- X Q, W <- W Q
  launch_bsr_step<double>(bsr_H(ctx), MODE_SPMM, act, ld, st.X, nullptr, st.W, nullptr, 1.0, 0.0, 0.0, 0.0, s);
  PFE_TRY(check_launch(ctx, "H X"));
  st.matvecs += act;
  {
    // A = X^T H X is symmetric: only the upper tiles are computed (half the flops), then mirrored
    RESERVE(double, gw, ctx->w_gram, gram_work(n, act, act, true));
    launch_gram(n, act, act, st.X, ld, st.W, ld, 1.0, 0.0, st.A, act, true, gw, s);
  }
  int lw = 0;
  if (G1) {
    // the second CholQR2 pass folded in: A c = theta G1 c with c^T G1 c = 1, so X1 C is orthonormal
    PFE_SOLVER_TRY(ctx, cusolverDnDsygvd_bufferSize(ctx->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                                    CUBLAS_FILL_MODE_UPPER, act, st.A, act, G1, act, st.resid2, &lw));
    RESERVE(double, work, ctx->w_cs_work, (size_t)std::max(lw, 1));
    PFE_SOLVER_TRY(ctx, cusolverDnDsygvd(ctx->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                         CUBLAS_FILL_MODE_UPPER, act, st.A, act, G1, act, st.evals, work, lw, st.info));
  } else {
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, act,
                                                    st.A, act, st.resid2, &lw));
    RESERVE(double, work, ctx->w_cs_work, (size_t)std::max(lw, 1));
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, act, st.A, act,
                                         st.evals, work, lw, st.info));
  }
  launch_update(n, act, act, st.X, ld, st.A, act, 1.0, 0.0, st.Y, ld, s);
  std::swap(st.X, st.Y);
  // W = H X again on the rotated block: one BSR product instead of the n x q x q update W <- W Q
  launch_bsr_step<double>(bsr_H(ctx), MODE_SPMM, act, ld, st.X, nullptr, st.W, nullptr, 1.0, 0.0, 0.0, 0.0, s);
  st.matvecs += act;
  launch_col_resid2(n, act, st.W, st.X, ld, st.evals, st.resid2, st.red, s);
  PFE_TRY(check_launch(ctx, "residuals"));
  cudaEventRecord(st.ev[3], s);
  int hinfo = 0;
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(st.hth.data(), st.evals, sizeof(double) * act, cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(st.hr2.data(), st.resid2, sizeof(double) * act, cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, st.info, sizeof(int), cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (hinfo != 0)
    return pfe_fail(ctx, PFE_E_CUDA, std::string(G1 ? "cusolverDnDsygvd" : "cusolverDnDsyevd") + " failed (info " +
                                         std::to_string(hinfo) + ")");
  float ms = 0;
  if (st.timed_filter) {
    cudaEventElapsedTime(&ms, st.ev[0], st.ev[1]);
    st.t_filter += ms * 1e-3;
  }
  if (st.timed32) {
    cudaEventElapsedTime(&ms, st.ev32[0], st.ev32[1]);
    st.t_filter32 += ms * 1e-3;
    st.timed32 = false;
  }
  cudaEventElapsedTime(&ms, st.ev[1], st.ev[2]);
  st.t_orth += ms * 1e-3;
  cudaEventElapsedTime(&ms, st.ev[2], st.ev[3]);
  st.t_rr += ms * 1e-3;
  const double lmax = ctx->lmax, tol = ctx->p_tol;

  // ---- convergence bookkeeping.  Converged: r <= tol.  An unconverged pair blocks termination
  // only when its residual interval [theta - r, theta + r] lies inside [a, b]: the Krylov-Weinstein
  // bound then places a not yet locked eigenvalue in the interval.  Other unconverged Ritz values
  // in [a, b] can be mixtures of eigenvectors from both sides and never converge.
  std::vector<double> rr(act);
  int count_in = 0, unconv_in = 0;
  for (double lv : st.lockLam)
    if (lv >= ctx->a && lv <= ctx->b) ++count_in;
  for (int32_t j = 0; j < act; ++j) {
    rr[j] = std::sqrt(std::max(st.hr2[j], 0.0)) / lmax;
    if (!std::isfinite(st.hth[j]) || !std::isfinite(rr[j]))
      return pfe_fail(ctx, PFE_E_BREAKDOWN, "non-finite Ritz value or residual");
    if (st.hth[j] > lmax * (1.0 + 1e-12)) return pfe_fail(ctx, PFE_E_BOUND, "a Ritz value exceeds the lambda_max bound");
    const double rabs = rr[j] * lmax;
    if (rr[j] <= tol) {
      if (st.hth[j] >= ctx->a && st.hth[j] <= ctx->b) ++count_in;
    } else if (st.hth[j] - rabs >= ctx->a && st.hth[j] + rabs <= ctx->b) {
      ++unconv_in;
    }
  }
  // ---- lock converged pairs and compact the active block.  Mixed precision: the kept pairs are
  // ordered [residual <= hand-over tolerance (FP64 filter) | the rest (FP32 filter)], the FP64
  // group padded to a multiple of 4 columns so that the FP32 group starts 16-byte aligned.
  std::vector<int32_t> lock_cols, keep_cols, keep32;
  for (int32_t j = 0; j < act; ++j) {
    if (rr[j] <= tol && st.nl + (int32_t)lock_cols.size() < q) lock_cols.push_back(j);
    else if (st.fp32 && rr[j] > ctx->p_refine_tol) keep32.push_back(j);
    else keep_cols.push_back(j);
  }
  if (st.fp32) {
    while (keep_cols.size() % 4 != 0 && !keep32.empty()) {
      keep_cols.push_back(keep32.front());
      keep32.erase(keep32.begin());
    }
    st.k64 = (int32_t)keep_cols.size();
    keep_cols.insert(keep_cols.end(), keep32.begin(), keep32.end());
  }
  const bool reorder = st.fp32 && !keep32.empty();
  if (!lock_cols.empty() || reorder) {
    if (!lock_cols.empty()) {
      PFE_CUDA_TRY(ctx, cudaMemcpyAsync(st.idx, lock_cols.data(), sizeof(int32_t) * lock_cols.size(),
                                        cudaMemcpyHostToDevice, s));
      launch_gather_cols(n, (int32_t)lock_cols.size(), st.X, ld, st.L + st.nl, ld, st.idx, s);
      for (int32_t j : lock_cols) {
        st.lockLam.push_back(st.hth[j]);
        st.lockRes.push_back(rr[j]);
      }
      st.nl += (int32_t)lock_cols.size();
      PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // st.idx is reused below
    }
    if (!keep_cols.empty()) {
      PFE_CUDA_TRY(ctx, cudaMemcpyAsync(st.idx, keep_cols.data(), sizeof(int32_t) * keep_cols.size(),
                                        cudaMemcpyHostToDevice, s));
      launch_gather_cols(n, (int32_t)keep_cols.size(), st.X, ld, st.Y, ld, st.idx, s);
      std::swap(st.X, st.Y);
      if (st.defect) {  // W = H X follows the kept columns (the next defect filter reads it)
        launch_gather_cols(n, (int32_t)keep_cols.size(), st.W, ld, st.T0, ld, st.idx, s);
        std::swap(st.W, st.T0);
      }
    }
    PFE_TRY(check_launch(ctx, "locking"));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // the host index vectors must outlive the copies
  }
  if (st.defect) {
    st.theta_act.clear();
    if (!lock_cols.empty() || reorder)
      for (int32_t j : keep_cols) st.theta_act.push_back(st.hth[j]);
    else
      st.theta_act.assign(st.hth.begin(), st.hth.begin() + act);
  }
  st.act = (int32_t)keep_cols.size();
  if ((unconv_in == 0 && count_in == st.prev_count && st.it >= 2) || st.act == 0) {
    st.result = (count_in >= q) ? PFE_E_CAPACITY : PFE_OK;
    st.done = true;
  } else if (st.it >= ctx->p_max_iters) {
    st.result = PFE_E_NOCONV;
    st.done = true;
  }
  st.prev_count = count_in;
  return PFE_OK;
}

pfe_status solve_finish(pfe_ctx *ctx, int32_t *n_found) {
  SolveState &st = ctx->solve;
  const double lmax = ctx->lmax;
  std::vector<int32_t> ord;
  for (int32_t l = 0; l < st.nl; ++l)
    if (st.lockLam[l] >= ctx->a && st.lockLam[l] <= ctx->b) ord.push_back(l);
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return st.lockLam[x] < st.lockLam[y]; });
  ctx->result_cols = ord;
  ctx->result_lam.clear();
  ctx->result_res.clear();
  double maxres = 0.0;
  for (int32_t l : ord) {
    ctx->result_lam.push_back(st.lockLam[l]);
    ctx->result_res.push_back(st.lockRes[l] * lmax);
    maxres = std::max(maxres, st.lockRes[l]);
  }
  ctx->n_found = (int32_t)ord.size();
  ctx->has_result = true;
  pfe_stats &o = ctx->stats;
  o.iterations = st.it;
  o.width = st.q;
  o.degree = ctx->m;
  o.n_found = ctx->n_found;
  o.matvecs = st.matvecs;
  o.lambda_max = lmax;
  o.count_estimate = ctx->has_count ? ctx->count_est : -1.0;
  o.window_estimate = st.window_est;
  o.seconds_filter = st.t_filter;
  o.seconds_filter_f32 = st.t_filter32;
  o.seconds_orth = st.t_orth;
  o.seconds_rr = st.t_rr;
  o.max_residual = maxres;
  o.fp64_sweeps = st.fp64_sweeps;
  o.cholqr_shifts = ctx->shift_count;
  o.status = (int32_t)st.result;
  o.kernel_launches = launch_count() - ctx->launch_base;
  o.filter_launches = st.f_launch;
  o.filter_col_steps = st.f_cols64;
  o.filter_col_steps_f32 = st.f_cols32;
  o.filter_col_steps_forced = st.f_cols_forced;
  o.filter_shape_f64 = st.f_cols64 > 0 ? step_last_variant(0) : -1;
  o.filter_shape_f32 = st.f_cols32 > 0 ? step_last_variant(1) : -1;
  o.seconds_total = now_s() - st.t_start;
  for (int e = 0; e < 4; ++e)
    if (st.ev[e]) {
      cudaEventDestroy(st.ev[e]);
      st.ev[e] = nullptr;
    }
  for (int e = 0; e < 2; ++e)
    if (st.ev32[e]) {
      cudaEventDestroy(st.ev32[e]);
      st.ev32[e] = nullptr;
    }
  if (n_found) *n_found = ctx->n_found;
  if (st.result == PFE_E_CAPACITY) return pfe_fail(ctx, st.result, "every Ritz vector lies in [a, b]: raise PFE_P_WIDTH");
  if (st.result == PFE_E_NOCONV)
    return pfe_fail(ctx, st.result, st.it >= ctx->p_max_iters ? "iteration limit reached" : "solve ended before convergence");
  return PFE_OK;
}

// ---------------------------------------------------------------- batched filter (host side)
// fn(i) for i in [0, ns) from up to nthreads host threads (0: min(ns, hardware threads, 16)), each
// bound to the device; every sample is touched by exactly one thread.
template <typename F>
void for_each_sample(int device, int32_t ns, int32_t nthreads, F &&fn) {
  int32_t nt = nthreads;
  if (nt <= 0) nt = (int32_t)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
  nt = std::min(nt, ns);
  if (nt <= 1) {
    for (int32_t i = 0; i < ns; ++i) fn(i);
    return;
  }
  std::atomic<int32_t> next{0};
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int32_t t = 0; t < nt; ++t)
    pool.emplace_back([&] {
      cudaSetDevice(device);
      for (int32_t i = next.fetch_add(1); i < ns; i = next.fetch_add(1)) fn(i);
    });
  for (auto &th : pool) th.join();
}

struct BatchPlan {
  DBuf desc, total;
  std::vector<BatchDesc> h;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t m_max = 0, cpl = 2, blocks = 0;
  cudaStream_t stream = nullptr;  // the batch's own stream (graphs cannot be captured on the legacy stream)
  cudaEvent_t e0 = nullptr, e1 = nullptr, done_ev = nullptr;
  std::vector<cudaEvent_t> ready;  // per sample: its stream's work before the batched filter
};

void batch_plan_free(BatchPlan *p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->e0) cudaEventDestroy(p->e0);
  if (p->e1) cudaEventDestroy(p->e1);
  if (p->done_ev) cudaEventDestroy(p->done_ev);
  for (cudaEvent_t e : p->ready)
    if (e) cudaEventDestroy(e);
  if (p->stream) {
    cudaStreamSynchronize(p->stream);
    cudaStreamDestroy(p->stream);
  }
  dbuf_free(p->desc);
  dbuf_free(p->total);
  *p = BatchPlan{};
}

// Refresh the descriptors of the FP64 samples that are still iterating; returns the item count.
int64_t batch_refresh(pfe_ctx **ctxs, int32_t ns, const std::vector<pfe_status> &status, BatchPlan *p) {
  int64_t items = 0;
  p->h.resize(ns);
  for (int32_t i = 0; i < ns; ++i) {
    pfe_ctx *c = ctxs[i];
    const SolveState &st = c->solve;
    BatchDesc &d = p->h[i];
    const bool live = status[i] == PFE_OK && !st.done && st.use64;
    d.rp = c->rp.as<int32_t>();
    d.ci = c->ci.as<int32_t>();
    d.vals = c->Hs64.as<double>();
    const bool r1 = c->p_rank1 && c->r1_state == 1;
    d.rp1 = r1 ? c->r1_rp.as<int32_t>() : nullptr;
    d.ci1 = r1 ? c->r1_ci.as<int32_t>() : nullptr;
    d.u = r1 ? c->r1_u64.as<double>() : nullptr;
    d.dg = r1 ? c->r1_dg64.as<double>() : nullptr;
    d.X = st.X;
    d.b0 = st.T0;
    d.b1 = st.T1;
    d.Y = st.Y;
    d.coef = c->dcoef.as<double>();
    d.ld = st.ld;
    d.n_atoms = c->N;
    d.k = live ? st.act : 0;
    d.m = live ? c->m : 0;
    d.nchunk = (d.k + 32 * p->cpl - 1) / (32 * p->cpl);
    d.item_begin = items;
    items += (int64_t)d.n_atoms * d.nchunk;
  }
  return items;
}

pfe_status batch_upload(pfe_ctx *c0, BatchPlan *p, int64_t items) {
  cudaStream_t s = p->stream;
  PFE_CUDA_TRY(c0, cudaMemcpyAsync(p->desc.p, p->h.data(), sizeof(BatchDesc) * p->h.size(), cudaMemcpyHostToDevice, s));
  PFE_CUDA_TRY(c0, cudaMemcpyAsync(p->total.p, &items, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  PFE_CUDA_TRY(c0, cudaStreamSynchronize(s));  // the host copies must outlive the transfers
  return PFE_OK;
}

pfe_status batch_plan_init(pfe_ctx *c0, pfe_ctx **ctxs, int32_t ns, const std::vector<pfe_status> &status,
                           BatchPlan *p) {
  PFE_CUDA_TRY(c0, cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
  cudaStream_t s = p->stream;
  for (int32_t i = 0; i < ns; ++i) {
    if (status[i] != PFE_OK) continue;
    pfe_ctx *c = ctxs[i];
    // coefficients on the device (read by the batched kernel)
    if (dbuf_reserve(c->dcoef, sizeof(double) * (c->m + 1)) != cudaSuccess)
      return pfe_fail(c0, PFE_E_NOMEM, "coefficient buffer");
    PFE_CUDA_TRY(c0, cudaMemcpy(c->dcoef.p, c->coef.data(), sizeof(double) * (c->m + 1), cudaMemcpyHostToDevice));
    p->m_max = std::max(p->m_max, c->m);
    PFE_CUDA_TRY(c0, cudaStreamSynchronize(c->stream));  // set-up work of every sample is complete
  }
  if (dbuf_reserve(p->desc, sizeof(BatchDesc) * ns) != cudaSuccess || dbuf_reserve(p->total, sizeof(int64_t)) != cudaSuccess)
    return pfe_fail(c0, PFE_E_NOMEM, "batch descriptors");
  PFE_CUDA_TRY(c0, cudaEventCreate(&p->e0));
  PFE_CUDA_TRY(c0, cudaEventCreate(&p->e1));
  PFE_CUDA_TRY(c0, cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming));
  int sms = 0;
  PFE_CUDA_TRY(c0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device));
  // autotuner: columns per warp (32 or 64) x persistent blocks per SM, timed on steps 0 and 1
  // (they write only scratch buffers), best of two trials each
  float best = 1e30f;
  int best_cpl = 2, best_blocks = sms * 8;
  if (p->m_max >= 2) {
    for (int cpl : {1, 2})
      for (int bps : {4, 8, 16}) {
        p->cpl = cpl;
        const int64_t items = batch_refresh(ctxs, ns, status, p);
        if (items == 0) continue;
        PFE_TRY(batch_upload(c0, p, items));
        float t_best = 1e30f;
        for (int trial = 0; trial < 2; ++trial) {
          cudaEventRecord(p->e0, s);
          launch_batch_step(cpl, sms * bps, p->desc.as<BatchDesc>(), ns, p->total.as<int64_t>(), 0, s);
          launch_batch_step(cpl, sms * bps, p->desc.as<BatchDesc>(), ns, p->total.as<int64_t>(), 1, s);
          cudaEventRecord(p->e1, s);
          PFE_CUDA_TRY(c0, cudaEventSynchronize(p->e1));
          float ms = 0;
          cudaEventElapsedTime(&ms, p->e0, p->e1);
          t_best = std::min(t_best, ms);
        }
        PFE_TRY(check_launch(c0, "batch autotune"));
        if (t_best < best) {
          best = t_best;
          best_cpl = cpl;
          best_blocks = sms * bps;
        }
      }
  }
  p->cpl = best_cpl;
  p->blocks = best_blocks;
  c0->tuned_cpl = best_cpl;
  c0->tuned_blocks = best_blocks;
  // capture the m_max steps of one filter application as a CUDA graph
  if (p->m_max > 0) {
    PFE_CUDA_TRY(c0, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int32_t j = 0; j < p->m_max; ++j)
      launch_batch_step(p->cpl, p->blocks, p->desc.as<BatchDesc>(), ns, p->total.as<int64_t>(), j, s);
    cudaError_t ce = cudaStreamEndCapture(s, &p->graph);
    if (ce != cudaSuccess) return pfe_fail(c0, PFE_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    PFE_CUDA_TRY(c0, cudaGraphInstantiate(&p->exec, p->graph, 0));
  }
  return PFE_OK;
}

// One filter application for every FP64 sample: refresh descriptors, replay the graph.
pfe_status batch_filter(pfe_ctx *c0, pfe_ctx **ctxs, int32_t ns, const std::vector<pfe_status> &status, BatchPlan *p,
                        float *ms) {
  cudaStream_t s = p->stream;
  *ms = 0.f;
  const int64_t items = batch_refresh(ctxs, ns, status, p);
  for (int32_t i = 0; i < ns; ++i) {
    const BatchDesc &d = p->h[i];
    if (d.k == 0) continue;
    SolveState &st = ctxs[i]->solve;
    st.was64 = true;
    st.f_launch += std::max(d.m, 1);
    st.f_cols64 += (int64_t)d.k * std::max(d.m, 1);
    st.matvecs += (int64_t)d.k * d.m;
    ++st.fp64_sweeps;
    // degree 0: y = g0 x (no Chebyshev step)
    if (d.m == 0) launch_axpby<double>(ctxs[i]->n, d.k, ctxs[i]->coef[0], st.X, st.ld, 0.0, st.Y, st.ld, ctxs[i]->stream);
  }
  if (items > 0 && p->exec) {
    // the graph reads every FP64 sample's block: wait for the work queued on the samples' streams
    if (p->ready.size() != (size_t)ns) p->ready.assign(ns, nullptr);
    for (int32_t i = 0; i < ns; ++i) {
      if (p->h[i].k == 0) continue;
      if (!p->ready[i]) PFE_CUDA_TRY(c0, cudaEventCreateWithFlags(&p->ready[i], cudaEventDisableTiming));
      PFE_CUDA_TRY(c0, cudaEventRecord(p->ready[i], ctxs[i]->stream));
      PFE_CUDA_TRY(c0, cudaStreamWaitEvent(s, p->ready[i], 0));
    }
    PFE_TRY(batch_upload(c0, p, items));
    cudaEventRecord(p->e0, s);
    PFE_CUDA_TRY(c0, cudaGraphLaunch(p->exec, s));
    cudaEventRecord(p->e1, s);
    PFE_CUDA_TRY(c0, cudaEventSynchronize(p->e1));
    cudaEventElapsedTime(ms, p->e0, p->e1);
    count_launches(p->m_max);
  }
  cudaEventRecord(p->done_ev, s);
  return check_launch(c0, "batched filter");
}

}  // namespace

namespace pfe {
pfe_status solver_ensure_filter(pfe_ctx *ctx) { return ensure_filter(ctx); }
pfe_status solver_ensure_hs(pfe_ctx *ctx, bool need32) { return ensure_hs(ctx, need32); }
pfe_status solver_count(pfe_ctx *ctx) { return count_estimate(ctx); }
pfe_status solver_window(pfe_ctx *ctx, double *out) { return window_estimate(ctx, out); }
pfe_status solver_cholqr2(pfe_ctx *ctx, double *Y, double *tmp, int32_t k, int64_t ld, double **result, bool *shifted) {
  return cholqr2(ctx, Y, tmp, k, ld, result, shifted);
}
pfe_status solver_filter64(pfe_ctx *ctx, int32_t k, int64_t ld, const double *X, double *Y, double *b0, double *b1) {
  return run_filter<double>(ctx, bsr_Hs64(ctx), ctx->coef.data(), ctx->m, k, ld, X, Y, b0, b1, ctx->stream);
}
pfe_status solver_filter64_rows(pfe_ctx *ctx, const double *coef, int32_t m, int32_t k, int64_t ld, const double *X,
                                double *Y, double *b0, double *b1, cudaStream_t s, bool tune) {
  return run_filter<double>(ctx, bsr_Hs64(ctx), coef, m, k, ld, X, Y, b0, b1, s, tune);
}
double solver_now() { return now_s(); }
pfe_status solver_ensure_lmax(pfe_ctx *ctx) { return ensure_lmax(ctx); }
Bsr<double> solver_bsr_H(const pfe_ctx *ctx) { return bsr_H(ctx); }
Bsr<double> solver_bsr_Hs64(const pfe_ctx *ctx) { return bsr_Hs64(ctx); }
}  // namespace pfe

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

pfe_status pfe_springs_to_bsr(int32_t n_atoms, int64_t nbonds, const int32_t *bi, const int32_t *bj, const double *k,
                              const double *rhat, int64_t cap_nnzb, int32_t *row_ptr, int32_t *col_idx, double *vals,
                              int64_t *nnzb) {
  if (n_atoms < 1 || nbonds < 0 || !nnzb) return PFE_E_ARG;
  if (nbonds > 0 && (!bi || !bj || !k || !rhat)) return PFE_E_ARG;
  for (int64_t e = 0; e < nbonds; ++e) {
    if (bi[e] < 0 || bi[e] >= n_atoms || bj[e] < 0 || bj[e] >= n_atoms || bi[e] == bj[e]) return PFE_E_ARG;
    if (!std::isfinite(k[e]) || !std::isfinite(rhat[3 * e]) || !std::isfinite(rhat[3 * e + 1]) ||
        !std::isfinite(rhat[3 * e + 2]))
      return PFE_E_ARG;
  }
  // neighbour lists (both directions), sorted by (neighbour, bond)
  std::vector<int64_t> off((size_t)n_atoms + 1, 0);
  for (int64_t e = 0; e < nbonds; ++e) {
    ++off[bi[e] + 1];
    ++off[bj[e] + 1];
  }
  for (int32_t i = 0; i < n_atoms; ++i) off[i + 1] += off[i];
  std::vector<std::pair<int32_t, int64_t>> nb((size_t)off[n_atoms]);
  {
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (int64_t e = 0; e < nbonds; ++e) {
      nb[pos[bi[e]]++] = {bj[e], e};
      nb[pos[bj[e]]++] = {bi[e], e};
    }
  }
  int64_t total = 0;
  for (int32_t i = 0; i < n_atoms; ++i) {
    std::sort(nb.begin() + off[i], nb.begin() + off[i + 1]);
    int64_t uniq = 0;
    for (int64_t t = off[i]; t < off[i + 1]; ++t)
      if (t == off[i] || nb[t].first != nb[t - 1].first) ++uniq;
    total += uniq + 1;
  }
  *nnzb = total;
  if (total > INT32_MAX) return PFE_E_ARG;
  if (cap_nnzb < total || !row_ptr || !col_idx || !vals) return PFE_E_CAPACITY;
  int64_t p = 0;
  auto rr = [&](int64_t e, int a, int b) {  // r_a r_b, symmetric in (a, b) bit for bit
    const double *r = rhat + 3 * e;
    return a <= b ? r[a] * r[b] : r[b] * r[a];
  };
  for (int32_t i = 0; i < n_atoms; ++i) {
    row_ptr[i] = (int32_t)p;
    double D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t t = off[i]; t < off[i + 1]; ++t)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) D[3 * a + b] += k[nb[t].second] * rr(nb[t].second, a, b);
    bool diag_done = false;
    int64_t t = off[i];
    while (t <= off[i + 1]) {
      const bool end = (t == off[i + 1]);
      if (!diag_done && (end || nb[t].first > i)) {
        col_idx[p] = i;
        std::memcpy(vals + 9 * p, D, sizeof(D));
        ++p;
        diag_done = true;
      }
      if (end) break;
      const int32_t j = nb[t].first;
      double B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      while (t < off[i + 1] && nb[t].first == j) {
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) B[3 * a + b] -= k[nb[t].second] * rr(nb[t].second, a, b);
        ++t;
      }
      col_idx[p] = j;
      std::memcpy(vals + 9 * p, B, sizeof(B));
      ++p;
    }
  }
  row_ptr[n_atoms] = (int32_t)p;
  return PFE_OK;
}

pfe_status pfe_create(pfe_ctx **out, int32_t n_atoms, int64_t nnzb, const int32_t *row_ptr, const int32_t *col_idx,
                      const double *vals, const double *masses, uint32_t flags, void *cuda_stream) {
  if (!out) return PFE_E_ARG;
  *out = nullptr;
  if (n_atoms < 1 || nnzb < n_atoms || nnzb > INT32_MAX || !row_ptr || !col_idx || !vals) return PFE_E_ARG;
  const bool dev = (flags & PFE_DEVICE_PTRS) != 0;
  std::vector<int32_t> rp((size_t)n_atoms + 1), ci((size_t)nnzb);
  std::vector<double> dv((size_t)9 * nnzb), ms;
  auto fetch = [&](void *dst, const void *src, size_t bytes) -> bool {
    if (!dev) {
      std::memcpy(dst, src, bytes);
      return true;
    }
    return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
  };
  if (!fetch(rp.data(), row_ptr, rp.size() * 4) || !fetch(ci.data(), col_idx, ci.size() * 4) ||
      !fetch(dv.data(), vals, dv.size() * 8))
    return PFE_E_CUDA;
  if (masses) {
    ms.resize((size_t)n_atoms);
    if (!fetch(ms.data(), masses, ms.size() * 8)) return PFE_E_CUDA;
    for (double m : ms)
      if (!(m > 0.0) || !std::isfinite(m)) return PFE_E_ARG;
  }
  // structure checks
  if (rp[0] != 0 || rp[n_atoms] != nnzb) return PFE_E_ARG;
  double vmax = 0.0;
  for (int32_t i = 0; i < n_atoms; ++i) {
    if (rp[i + 1] < rp[i]) return PFE_E_ARG;
    bool has_diag = false;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= n_atoms) return PFE_E_ARG;
      if (p > rp[i] && ci[p] <= ci[p - 1]) return PFE_E_ARG;
      if (ci[p] == i) has_diag = true;
    }
    if (!has_diag) return PFE_E_ARG;
  }
  for (double v : dv) {
    if (!std::isfinite(v)) return PFE_E_ARG;
    vmax = std::max(vmax, std::fabs(v));
  }
  if (!(flags & PFE_SKIP_SYM_CHECK)) {
    const double tol = 1e-12 * vmax;
    for (int32_t i = 0; i < n_atoms; ++i)
      for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        const int32_t j = ci[p];
        if (j < i) continue;
        const int32_t *lo = ci.data() + rp[j], *hi = ci.data() + rp[j + 1];
        const int32_t *f = std::lower_bound(lo, hi, i);
        if (f == hi || *f != i) return PFE_E_NOTSYM;
        const int64_t q = f - ci.data();
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            if (std::fabs(dv[9 * (size_t)p + 3 * a + b] - dv[9 * (size_t)q + 3 * b + a]) > tol) return PFE_E_NOTSYM;
      }
  }
  pfe_ctx *ctx = new (std::nothrow) pfe_ctx();
  if (!ctx) return PFE_E_NOMEM;
  ctx->N = n_atoms;
  ctx->n = 3 * (int64_t)n_atoms;
  ctx->launch_base = launch_count();
  ctx->nnzb = nnzb;
  ctx->has_mass = masses != nullptr;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  auto bail = [&](pfe_status s) {
    pfe_destroy(ctx);
    return s;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(PFE_E_CUDA);
  if (cublasCreate(&ctx->blas) != CUBLAS_STATUS_SUCCESS) return bail(PFE_E_CUDA);
  if (cublasSetStream(ctx->blas, ctx->stream) != CUBLAS_STATUS_SUCCESS) return bail(PFE_E_CUDA);
  if (cusolverDnCreate(&ctx->solver) != CUSOLVER_STATUS_SUCCESS) return bail(PFE_E_CUDA);
  if (cusolverDnSetStream(ctx->solver, ctx->stream) != CUSOLVER_STATUS_SUCCESS) return bail(PFE_E_CUDA);
  DBuf delta;
  if (dbuf_reserve(ctx->rp, rp.size() * 4) || dbuf_reserve(ctx->ci, ci.size() * 4) ||
      dbuf_reserve(ctx->H, dv.size() * 8) || dbuf_reserve(delta, dv.size() * 8))
    return bail(PFE_E_NOMEM);
  cudaStream_t s = ctx->stream;
  if (cudaMemcpyAsync(ctx->rp.p, rp.data(), rp.size() * 4, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(ctx->ci.p, ci.data(), ci.size() * 4, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(masses ? delta.p : ctx->H.p, dv.data(), dv.size() * 8, cudaMemcpyHostToDevice, s)) {
    dbuf_free(delta);
    return bail(PFE_E_CUDA);
  }
  if (masses) {
    if (dbuf_reserve(ctx->mass, ms.size() * 8) ||
        cudaMemcpyAsync(ctx->mass.p, ms.data(), ms.size() * 8, cudaMemcpyHostToDevice, s)) {
      dbuf_free(delta);
      return bail(PFE_E_NOMEM);
    }
    launch_mass_weight(n_atoms, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), delta.as<double>(), ctx->mass.as<double>(),
                       ctx->H.as<double>(), s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  dbuf_free(delta);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return bail(PFE_E_CUDA);
  *out = ctx;
  return PFE_OK;
}

void pfe_destroy(pfe_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  DBuf *bufs[] = {&ctx->rp, &ctx->ci, &ctx->H, &ctx->mass, &ctx->Hs64, &ctx->Hs32, &ctx->L, &ctx->w_X, &ctx->w_Y,
                  &ctx->w_W, &ctx->w_T0, &ctx->w_T1, &ctx->w_T2, &ctx->w_small, &ctx->w_small2, &ctx->w_red,
                  &ctx->w_idx, &ctx->w_cs_work, &ctx->w_info, &ctx->w_f32a, &ctx->w_f32b, &ctx->w_f32c,
                  &ctx->w_f32d, &ctx->w_ckpt, &ctx->w_rr, &ctx->w_gram,
                  &ctx->w_bks[0], &ctx->w_bks[1], &ctx->w_bks[2], &ctx->w_bks[3], &ctx->w_bks[4],
                  &ctx->r1_rp, &ctx->r1_ci, &ctx->r1_u64, &ctx->r1_dg64, &ctx->r1_u32, &ctx->r1_dg32,
                  &ctx->r1_flag, &ctx->w_slice[0], &ctx->w_slice[1], &ctx->w_f32e, &ctx->w_defect, &ctx->w_tau,
                  &ctx->t_ptr, &ctx->t_atoms, &ctx->t_slot1, &ctx->t_self};
  for (DBuf *b : bufs) dbuf_free(*b);
  for (int e = 0; e < 4; ++e)
    if (ctx->solve.ev[e]) cudaEventDestroy(ctx->solve.ev[e]);
  for (int e = 0; e < 2; ++e)
    if (ctx->solve.ev32[e]) cudaEventDestroy(ctx->solve.ev32[e]);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->blas) cublasDestroy(ctx->blas);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  delete ctx;
}

const char *pfe_last_error(const pfe_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pfe_status pfe_set_param(pfe_ctx *ctx, int key, double v) {
  if (!ctx) return PFE_E_ARG;
  if (!std::isfinite(v)) return pfe_fail(ctx, PFE_E_ARG, "parameter value must be finite");
  auto int_ok = [&](double lo) { return v >= lo && v == std::floor(v) && v < 2147483647.0; };
  switch (key) {
    case PFE_P_DEGREE:
      if (!int_ok(0)) return pfe_fail(ctx, PFE_E_ARG, "DEGREE must be an integer >= 0");
      ctx->p_degree = (int32_t)v;
      ctx->has_filter = false;
      break;
    case PFE_P_EPS_FRAC:
      if (!(v > 0)) return pfe_fail(ctx, PFE_E_ARG, "EPS_FRAC must be > 0");
      ctx->p_eps_frac = v;
      ctx->has_filter = false;
      break;
    case PFE_P_RATE:
      if (!(v > 0 && v < 1)) return pfe_fail(ctx, PFE_E_ARG, "RATE must be in (0, 1)");
      ctx->p_rate = v;
      ctx->has_filter = false;
      break;
    case PFE_P_DAMPING:
      if (!(v == 0 || v == 1 || v == 2)) return pfe_fail(ctx, PFE_E_ARG, "DAMPING must be 0, 1 or 2");
      ctx->p_damping = (int)v;
      ctx->has_filter = false;
      break;
    case PFE_P_WIDTH:
      if (!int_ok(0)) return pfe_fail(ctx, PFE_E_ARG, "WIDTH must be an integer >= 0");
      ctx->p_width = (int32_t)v;
      break;
    case PFE_P_WIDTH_FACTOR:
      if (!(v >= 1.0)) return pfe_fail(ctx, PFE_E_ARG, "WIDTH_FACTOR must be >= 1");
      ctx->p_width_factor = v;
      break;
    case PFE_P_TOL:
      if (!(v > 0)) return pfe_fail(ctx, PFE_E_ARG, "TOL must be > 0");
      ctx->p_tol = v;
      break;
    case PFE_P_PRECISION:
      if (!(v == 0 || v == 1 || v == 2)) return pfe_fail(ctx, PFE_E_ARG, "PRECISION must be 0, 1 or 2");
      ctx->p_precision = (int)v;
      break;
    case PFE_P_MAX_ITERS:
      if (!int_ok(1)) return pfe_fail(ctx, PFE_E_ARG, "MAX_ITERS must be an integer >= 1");
      ctx->p_max_iters = (int32_t)v;
      break;
    case PFE_P_SEED:
      if (!(v >= 0 && v == std::floor(v) && v < 9007199254740992.0)) return pfe_fail(ctx, PFE_E_ARG, "SEED must be a non-negative integer");
      ctx->p_seed = (uint64_t)v;
      ctx->has_count = false;
      if (ctx->p_lambda_max <= 0) ctx->has_lmax = ctx->has_filter = false;
      break;
    case PFE_P_LAMBDA_MAX:
      if (!(v >= 0)) return pfe_fail(ctx, PFE_E_ARG, "LAMBDA_MAX must be >= 0");
      ctx->p_lambda_max = v;
      ctx->has_lmax = ctx->has_filter = ctx->has_count = false;
      break;
    case PFE_P_LAMBDA_MIN:
      ctx->p_lambda_min = v;
      ctx->has_lmax = ctx->has_filter = ctx->has_count = false;
      break;
    case PFE_P_COUNT_M:
      if (!int_ok(1)) return pfe_fail(ctx, PFE_E_ARG, "COUNT_M must be an integer >= 1");
      ctx->p_count_m = (int32_t)v;
      ctx->has_count = false;
      break;
    case PFE_P_COUNT_DEGREE:
      if (!int_ok(0)) return pfe_fail(ctx, PFE_E_ARG, "COUNT_DEGREE must be an integer >= 0");
      ctx->p_count_degree = (int32_t)v;
      ctx->has_count = false;
      break;
    case PFE_P_LANCZOS_STEPS:
      if (!int_ok(1)) return pfe_fail(ctx, PFE_E_ARG, "LANCZOS_STEPS must be an integer >= 1");
      ctx->p_lanczos_steps = (int32_t)v;
      if (ctx->p_lambda_max <= 0) ctx->has_lmax = ctx->has_filter = ctx->has_count = false;
      break;
    case PFE_P_COUNT_DAMPING:
      if (!(v == 0 || v == 1 || v == 2)) return pfe_fail(ctx, PFE_E_ARG, "COUNT_DAMPING must be 0, 1 or 2");
      ctx->p_count_damping = (int)v;
      ctx->has_count = false;
      break;
    case PFE_P_MIN_WIDTH:
      if (!int_ok(1)) return pfe_fail(ctx, PFE_E_ARG, "MIN_WIDTH must be an integer >= 1");
      ctx->p_min_width = (int32_t)v;
      break;
    case PFE_P_REFINE_TOL:
      if (!(v > 0)) return pfe_fail(ctx, PFE_E_ARG, "REFINE_TOL must be > 0");
      ctx->p_refine_tol = v;
      break;
    case PFE_P_METHOD:
      if (!(v == 0 || v == 1)) return pfe_fail(ctx, PFE_E_ARG, "METHOD must be 0 or 1");
      ctx->p_method = (int)v;
      if (ctx->p_rate <= 0.0) ctx->has_filter = false;  // the default rate depends on the method
      break;
    case PFE_P_BLOCK:
      if (!int_ok(1) || v > 4096) return pfe_fail(ctx, PFE_E_ARG, "BLOCK must be an integer in [1, 4096]");
      ctx->p_block = (int32_t)v;
      break;
    case PFE_P_BASIS_FACTOR:
      if (!(v >= 1.25)) return pfe_fail(ctx, PFE_E_ARG, "BASIS_FACTOR must be >= 1.25");
      ctx->p_basis_factor = v;
      break;
    case PFE_P_BATCH_THREADS:
      if (!int_ok(0) || v > 256) return pfe_fail(ctx, PFE_E_ARG, "BATCH_THREADS must be an integer in [0, 256]");
      ctx->p_batch_threads = (int32_t)v;
      break;
    case PFE_P_FILTER:
      if (!(v == 0 || v == 1)) return pfe_fail(ctx, PFE_E_ARG, "FILTER must be 0 or 1");
      ctx->p_filter = (int)v;
      ctx->has_filter = false;
      break;
    case PFE_P_PHI:
      if (!(v > 0 && v < 1)) return pfe_fail(ctx, PFE_E_ARG, "PHI must be in (0, 1)");
      ctx->p_phi = v;
      ctx->has_filter = false;
      break;
    case PFE_P_DIRAC_CUT:
      if (!(v > 0 && v <= 1)) return pfe_fail(ctx, PFE_E_ARG, "DIRAC_CUT must be in (0, 1]");
      ctx->p_dirac_cut = v;
      break;
    case PFE_P_SLICE_TARGET:
      if (!int_ok(1)) return pfe_fail(ctx, PFE_E_ARG, "SLICE_TARGET must be an integer >= 1");
      ctx->p_slice_target = (int32_t)v;
      break;
    case PFE_P_OVERLAP:
      if (!(v == 0 || v == 1)) return pfe_fail(ctx, PFE_E_ARG, "OVERLAP must be 0 or 1");
      ctx->p_overlap = (int)v;
      break;
    case PFE_P_DEGREE_RULE:
      if (!(v == 0 || v == 1)) return pfe_fail(ctx, PFE_E_ARG, "DEGREE_RULE must be 0 or 1");
      ctx->p_degree_rule = (int)v;
      ctx->has_filter = false;
      break;
    case PFE_P_RANK1:
      if (!(v == 0 || v == 1)) return pfe_fail(ctx, PFE_E_ARG, "RANK1 must be 0 or 1");
      ctx->p_rank1 = (int)v;
      if (ctx->p_rank1 && ctx->r1_state == -1) ctx->hs_valid = false;  // build the form with the next filter
      break;
    case PFE_P_STEP_SHAPE_F64:
    case PFE_P_STEP_SHAPE_F32:
      if (!(v == -1 || (v >= 0 && v <= 11 && v == std::floor(v))))
        return pfe_fail(ctx, PFE_E_ARG, "STEP_SHAPE must be -1 (autotuned) or 0..11");
      set_step_variant(key == PFE_P_STEP_SHAPE_F32, (int)v);
      break;
    default:
      return pfe_fail(ctx, PFE_E_ARG, "unknown parameter key " + std::to_string(key));
  }
  return PFE_OK;
}

pfe_status pfe_get_param(const pfe_ctx *ctx, int key, double *v) {
  if (!ctx || !v) return PFE_E_ARG;
  switch (key) {
    case PFE_P_DEGREE: *v = ctx->p_degree; break;
    case PFE_P_EPS_FRAC: *v = ctx->p_eps_frac; break;
    case PFE_P_RATE: *v = ctx->rate_of(); break;
    case PFE_P_DAMPING: *v = ctx->p_damping; break;
    case PFE_P_WIDTH: *v = ctx->p_width; break;
    case PFE_P_WIDTH_FACTOR: *v = ctx->p_width_factor; break;
    case PFE_P_TOL: *v = ctx->p_tol; break;
    case PFE_P_PRECISION: *v = ctx->p_precision; break;
    case PFE_P_MAX_ITERS: *v = ctx->p_max_iters; break;
    case PFE_P_SEED: *v = (double)ctx->p_seed; break;
    case PFE_P_LAMBDA_MAX: *v = ctx->p_lambda_max; break;
    case PFE_P_LAMBDA_MIN: *v = ctx->p_lambda_min; break;
    case PFE_P_COUNT_M: *v = ctx->p_count_m; break;
    case PFE_P_COUNT_DEGREE: *v = ctx->p_count_degree; break;
    case PFE_P_LANCZOS_STEPS: *v = ctx->p_lanczos_steps; break;
    case PFE_P_COUNT_DAMPING: *v = ctx->p_count_damping; break;
    case PFE_P_MIN_WIDTH: *v = ctx->p_min_width; break;
    case PFE_P_REFINE_TOL: *v = ctx->p_refine_tol; break;
    case PFE_P_METHOD: *v = ctx->p_method; break;
    case PFE_P_BLOCK: *v = ctx->p_block; break;
    case PFE_P_BASIS_FACTOR: *v = ctx->p_basis_factor; break;
    case PFE_P_BATCH_THREADS: *v = ctx->p_batch_threads; break;
    case PFE_P_RANK1: *v = (ctx->p_rank1 && ctx->r1_state == 1) ? 1.0 : 0.0; break;
    case PFE_P_FILTER: *v = ctx->p_filter; break;
    case PFE_P_PHI: *v = ctx->p_phi; break;
    case PFE_P_DIRAC_CUT: *v = ctx->p_dirac_cut; break;
    case PFE_P_SLICE_TARGET: *v = ctx->p_slice_target; break;
    case PFE_P_OVERLAP: *v = ctx->p_overlap; break;
    case PFE_P_DEGREE_RULE: *v = ctx->p_degree_rule; break;
    case PFE_P_STEP_SHAPE_F64: *v = step_variant(0); break;
    case PFE_P_STEP_SHAPE_F32: *v = step_variant(1); break;
    default: return PFE_E_ARG;
  }
  return PFE_OK;
}

pfe_status pfe_set_interval(pfe_ctx *ctx, double a, double b) {
  if (!ctx) return PFE_E_ARG;
  if (!std::isfinite(a) || !std::isfinite(b) || !(a < b) || a < 0)
    return pfe_fail(ctx, PFE_E_ARG, "interval must satisfy 0 <= a < b");
  ctx->a = a;
  ctx->b = b;
  ctx->has_interval = true;
  ctx->has_filter = ctx->has_count = false;
  return PFE_OK;
}

pfe_status pfe_estimate(pfe_ctx *ctx, double *lambda_max, double *count_est) {
  if (!ctx) return PFE_E_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  PFE_TRY(ensure_lmax(ctx));
  if (lambda_max) *lambda_max = ctx->lmax;
  if (count_est) {
    if (ctx->has_interval) {
      PFE_TRY(count_estimate(ctx));
      *count_est = ctx->count_est;
    } else {
      *count_est = std::nan("");
    }
  }
  return PFE_OK;
}

pfe_status pfe_get_filter(pfe_ctx *ctx, int32_t cap, int32_t *m, double *coeffs, double *c, double *d) {
  if (!ctx) return PFE_E_ARG;
  PFE_TRY(ensure_filter(ctx));
  if (m) *m = ctx->m;
  if (c) *c = ctx->tc;
  if (d) *d = ctx->td;
  if (coeffs) {
    if (cap < ctx->m + 1) return pfe_fail(ctx, PFE_E_CAPACITY, "coefficient buffer too small");
    std::copy(ctx->coef.begin(), ctx->coef.end(), coeffs);
  }
  return PFE_OK;
}

pfe_status pfe_solve_begin(pfe_ctx *ctx) {
  if (!ctx) return PFE_E_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  if (ctx->p_method != 0)
    return pfe_fail(ctx, PFE_E_ARG, "the stepwise solve runs the filtered subspace iteration (METHOD 0)");
  ctx->solve.active = false;
  PFE_TRY(solve_setup(ctx));
  ctx->solve.active = true;
  return PFE_OK;
}

pfe_status pfe_solve_iterate(pfe_ctx *ctx, int32_t *done) {
  if (!ctx) return PFE_E_ARG;
  SolveState &st = ctx->solve;
  if (!st.active) return pfe_fail(ctx, PFE_E_STATE, "no stepwise solve in progress (pfe_solve_begin)");
  if (!st.done) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
    cudaEventRecord(st.ev[0], ctx->stream);
    pfe_status r = solve_filter(ctx);
    if (r == PFE_OK) r = solve_after_filter(ctx);
    if (r != PFE_OK) {
      st.active = false;
      return r;
    }
  }
  if (done) *done = st.done ? 1 : 0;
  return PFE_OK;
}

pfe_status pfe_solve_end(pfe_ctx *ctx, int32_t *n_found) {
  if (!ctx) return PFE_E_ARG;
  SolveState &st = ctx->solve;
  if (!st.active) return pfe_fail(ctx, PFE_E_STATE, "no stepwise solve in progress (pfe_solve_begin)");
  st.active = false;
  if (!st.done) {  // ended early: the pairs locked so far are the results
    st.result = PFE_E_NOCONV;
    st.done = true;
  }
  return solve_finish(ctx, n_found);
}

pfe_status pfe_solve(pfe_ctx *ctx, int32_t *n_found) {
  if (!ctx) return PFE_E_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  if (ctx->p_method == 1) return bks_solve(ctx, n_found);
  PFE_TRY(pfe_solve_begin(ctx));
  int32_t done = 0;
  while (!done) PFE_TRY(pfe_solve_iterate(ctx, &done));
  return pfe_solve_end(ctx, n_found);
}

pfe_status pfe_get_stats(const pfe_ctx *ctx, pfe_stats *st) {
  if (!ctx || !st) return PFE_E_ARG;
  *st = ctx->stats;
  st->active = st->locked = 0;
  const SolveState &ss = ctx->solve;
  if (ss.active) {  // a stepwise solve in progress
    st->iterations = ss.it;
    st->matvecs = ss.matvecs;
    st->width = ss.q;
    st->degree = ctx->m;
    st->active = ss.act;
    st->locked = ss.nl;
    st->kernel_launches = launch_count() - ctx->launch_base;
    st->cholqr_shifts = ctx->shift_count;
  }
  return PFE_OK;
}

pfe_status pfe_get_eigenpairs(pfe_ctx *ctx, int32_t cap, double *lambda, double *vecs, double *resid, uint32_t flags) {
  if (!ctx) return PFE_E_ARG;
  if (!ctx->has_result) return pfe_fail(ctx, PFE_E_STATE, "no solve results");
  const int32_t nf = ctx->n_found;
  if (cap < nf) return pfe_fail(ctx, PFE_E_CAPACITY, "output capacity below the number of eigenpairs found");
  if (lambda) std::copy(ctx->result_lam.begin(), ctx->result_lam.end(), lambda);
  if (resid) std::copy(ctx->result_res.begin(), ctx->result_res.end(), resid);
  if (vecs && nf > 0) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
    const int64_t n = ctx->n;
    cudaStream_t s = ctx->stream;
    const int64_t ldt = round_up(nf, 4);
    RESERVE(double, tmp, ctx->w_Y, (size_t)n * ldt);
    RESERVE(int32_t, idx, ctx->w_idx, (size_t)nf);
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(idx, ctx->result_cols.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
    launch_gather_cols(n, nf, ctx->L.as<double>(), ctx->ldq, tmp, ldt, idx, s);
    if (flags & PFE_DEVICE_PTRS) {
      launch_rowmajor_to_colmajor<double>(n, nf, tmp, ldt, vecs, n, s);
    } else {
      RESERVE(double, cm, ctx->w_W, (size_t)n * nf);
      launch_rowmajor_to_colmajor<double>(n, nf, tmp, ldt, cm, n, s);
      PFE_CUDA_TRY(ctx, cudaMemcpyAsync(vecs, cm, sizeof(double) * n * nf, cudaMemcpyDeviceToHost, s));
    }
    PFE_TRY(check_launch(ctx, "eigenvector export"));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  }
  return PFE_OK;
}

pfe_status pfe_filter_apply(pfe_ctx *ctx, int32_t m, const double *coeffs, int32_t k, const void *X, int64_t ldx,
                            void *Y, int64_t ldy, int dtype, void *stream) {
  if (!ctx) return PFE_E_ARG;
  if (k < 0 || (k > 0 && (!X || !Y)) || ldx < ctx->n || ldy < ctx->n || (dtype != PFE_F64 && dtype != PFE_F32))
    return pfe_fail(ctx, PFE_E_ARG, "filter_apply: bad arguments");
  if (coeffs && m < 0) return pfe_fail(ctx, PFE_E_ARG, "filter_apply: negative degree");
  if (k == 0) return PFE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  const double *cf = coeffs;
  if (!cf) {
    PFE_TRY(ensure_filter(ctx));
    cf = ctx->coef.data();
    m = ctx->m;
  }
  for (int32_t j = 0; j <= m; ++j)
    if (!std::isfinite(cf[j])) return pfe_fail(ctx, PFE_E_ARG, "filter_apply: non-finite coefficient");
  PFE_TRY(ensure_hs(ctx, dtype == PFE_F32));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
  if (s != ctx->stream) PFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // matrices built on ctx stream
  const int64_t n = ctx->n, ld = round_up(k, 4);
  const size_t big = (size_t)n * ld;
  if (dtype == PFE_F64) {
    RESERVE(double, Xr, ctx->w_X, big);
    RESERVE(double, Yr, ctx->w_Y, big);
    RESERVE(double, b0, ctx->w_T0, big);
    RESERVE(double, b1, ctx->w_T1, big);
    launch_colmajor_to_rowmajor<double>(n, k, static_cast<const double *>(X), ldx, Xr, ld, s);
    PFE_TRY(run_filter<double>(ctx, bsr_Hs64(ctx), cf, m, k, ld, Xr, Yr, b0, b1, s));
    launch_rowmajor_to_colmajor<double>(n, k, Yr, ld, static_cast<double *>(Y), ldy, s);
  } else {
    RESERVE(float, Xr, ctx->w_f32a, big);
    RESERVE(float, Yr, ctx->w_f32b, big);
    RESERVE(float, b0, ctx->w_f32c, big);
    RESERVE(float, b1, ctx->w_f32d, big);
    launch_colmajor_to_rowmajor<float>(n, k, static_cast<const float *>(X), ldx, Xr, ld, s);
    PFE_TRY(run_filter<float>(ctx, bsr_Hs32(ctx), cf, m, k, ld, Xr, Yr, b0, b1, s));
    launch_rowmajor_to_colmajor<float>(n, k, Yr, ld, static_cast<float *>(Y), ldy, s);
  }
  return check_launch(ctx, "filter_apply");
}

pfe_status pfe_filter_adjoint(pfe_ctx *ctx, int32_t m, const double *coeffs, int32_t k, const double *X, int64_t ldx,
                              const double *Ybar, int64_t ldyb, double *Xbar, int64_t ldxb, double *vals_bar,
                              void *stream) {
  if (!ctx) return PFE_E_ARG;
  if (k < 0 || (k > 0 && (!X || !Ybar || !Xbar)) || !vals_bar || ldx < ctx->n || ldyb < ctx->n || ldxb < ctx->n)
    return pfe_fail(ctx, PFE_E_ARG, "filter_adjoint: bad arguments");
  if (coeffs && m < 0) return pfe_fail(ctx, PFE_E_ARG, "filter_adjoint: negative degree");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  const double *cf = coeffs;
  if (!cf) {
    PFE_TRY(ensure_filter(ctx));
    cf = ctx->coef.data();
    m = ctx->m;
  }
  PFE_TRY(ensure_hs(ctx, false));
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
  if (s != ctx->stream) PFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  launch_zero<double>(vals_bar, 9 * ctx->nnzb, s);
  if (k == 0) return check_launch(ctx, "filter_adjoint");
  const int64_t n = ctx->n, ld = round_up(k, 2);
  const size_t vec = (size_t)n * ld;
  // checkpoint spacing ~ sqrt(m): checkpoints hold (t_j0, t_{j0+1}) for j0 = 0, S, 2S, ...
  const int32_t S = std::max<int32_t>(1, (int32_t)std::ceil(std::sqrt((double)std::max(m, 1))));
  const int32_t nseg = (m + S - 1) / S;
  // buffers: Xr, Ybr, adjoint segment of S + 2 vectors, forward segment of S + 1 vectors,
  // checkpoints 2 * nseg
  const size_t nvec = 2 + (size_t)(S + 2) + (size_t)(S + 1) + 2 * (size_t)std::max(nseg, 1);
  RESERVE(double, base, ctx->w_ckpt, vec * nvec);
  double *Xr = base, *Yb = base + vec, *aseg = base + 2 * vec;
  double *seg = aseg + (size_t)(S + 2) * vec;
  double *ck = seg + (size_t)(S + 1) * vec;
  launch_zero<double>(base, (int64_t)(vec * nvec), s);
  launch_colmajor_to_rowmajor<double>(n, k, X, ldx, Xr, ld, s);
  launch_colmajor_to_rowmajor<double>(n, k, Ybar, ldyb, Yb, ld, s);
  const Bsr<double> A = bsr_Hs64(ctx);
  const double two_over_d = 2.0 / ctx->td;
  auto tvec = [&](int32_t g, int which) { return ck + ((size_t)2 * g + which) * vec; };
  auto av = [&](int32_t q) { return aseg + (size_t)q * vec; };
  // forward pass: t_0 .. t_{m-1}, storing (t_j0, t_{j0+1}) at every segment start j0 = g S
  if (m >= 1) {
    double *tp = seg, *tc = seg + vec;  // rolling (t_{j-1}, t_j)
    launch_axpby<double>(n, k, 1.0, Xr, ld, 0.0, tp, ld, s);
    launch_bsr_step<double>(A, MODE_SPMM, k, ld, Xr, nullptr, tc, nullptr, 0.5, 0.0, 0.0, 0.0, s);
    launch_axpby<double>(n, k, 1.0, tp, ld, 0.0, tvec(0, 0), ld, s);
    launch_axpby<double>(n, k, 1.0, tc, ld, 0.0, tvec(0, 1), ld, s);
    for (int32_t j = 1; j + 1 < m; ++j) {
      // t_{j+1} = A t_j - t_{j-1}, written over t_{j-1}
      launch_bsr_step<double>(A, MODE_STEP, k, ld, tc, tp, tp, nullptr, 1.0, -1.0, 0.0, 0.0, s);
      std::swap(tp, tc);  // (tp, tc) = (t_j, t_{j+1})
      if (j % S == 0) {
        launch_axpby<double>(n, k, 1.0, tp, ld, 0.0, tvec(j / S, 0), ld, s);
        launch_axpby<double>(n, k, 1.0, tc, ld, 0.0, tvec(j / S, 1), ld, s);
      }
    }
    if (m - 1 >= 1 && (m - 1) % S == 0) launch_axpby<double>(n, k, 1.0, tc, ld, 0.0, tvec((m - 1) / S, 0), ld, s);
    PFE_TRY(check_launch(ctx, "adjoint forward"));
  }
  // reverse pass: a_m = g_m ybar, a_{m+1} = 0; a_j = A a_{j+1} - a_{j+2} + g_j ybar (j >= 1),
  // a_0 = A a_1 / 2 - a_2 + g_0 ybar; dL/dA += (2/d) a_{j+1} t_j^T (j >= 1) and (1/d) a_1 t_0^T.
  // Within the segment [j0, j1) the adjoint vectors a_{j0} .. a_{j1+1} sit in av(0) .. av(j1-j0+1),
  // and the segment's outer products are summed by one launch.
  if (m >= 1) {
    const int32_t jl0 = (nseg - 1) * S;
    launch_axpby<double>(n, k, cf[m], Yb, ld, 0.0, av(m - jl0), ld, s);  // a_m; a_{m+1} is zero
  }
  for (int32_t g = nseg - 1; g >= 0 && m >= 1; --g) {
    const int32_t j0 = g * S, j1 = std::min(m, j0 + S);  // this segment holds t_j0 .. t_{j1-1}
    // recompute the segment from its checkpoint
    launch_axpby<double>(n, k, 1.0, tvec(g, 0), ld, 0.0, seg, ld, s);
    if (j1 - j0 > 1) launch_axpby<double>(n, k, 1.0, tvec(g, 1), ld, 0.0, seg + vec, ld, s);
    for (int32_t j = j0 + 2; j < j1; ++j) {
      double *out = seg + (size_t)(j - j0) * vec;
      launch_bsr_step<double>(A, MODE_STEP, k, ld, seg + (size_t)(j - j0 - 1) * vec, seg + (size_t)(j - j0 - 2) * vec,
                              out, nullptr, 1.0, -1.0, 0.0, 0.0, s);
    }
    for (int32_t j = j1 - 1; j >= j0; --j)
      launch_bsr_step<double>(A, MODE_ADJ, k, ld, av(j - j0 + 1), av(j - j0 + 2), av(j - j0), Yb, j >= 1 ? 1.0 : 0.5,
                              -1.0, cf[j], 0.0, s);
    // sum_{j in [j0, j1)} alpha_j a_{j+1} t_j^T over the stored blocks
    launch_outer_accum_seg(A, ctx->nnzb, k, ld, j1 - j0, (int64_t)vec, av(1), seg, two_over_d * (j0 == 0 ? 0.5 : 1.0),
                           two_over_d, vals_bar, s);
    if (g > 0) {  // (a_{j0}, a_{j0+1}) become the next segment's (a_{j1'}, a_{j1'+1}), j1' = j0
      launch_axpby<double>(n, k, 1.0, av(1), ld, 0.0, av(S + 1), ld, s);
      launch_axpby<double>(n, k, 1.0, av(0), ld, 0.0, av(S), ld, s);
    }
  }
  double *an1 = av(0);  // a_0
  // a_0 = g_0 ybar for m == 0
  if (m == 0) launch_axpby<double>(n, k, cf[0], Yb, ld, 0.0, an1, ld, s);
  launch_rowmajor_to_colmajor<double>(n, k, an1, ld, Xbar, ldxb, s);
  return check_launch(ctx, "filter_adjoint");
}

pfe_status pfe_chain_springs(pfe_ctx *ctx, int64_t nbonds, const int32_t *bi, const int32_t *bj, const double *rhat,
                             const double *vals_bar, double *k_bar, double *m_bar, void *stream) {
  if (!ctx) return PFE_E_ARG;
  if (!ctx->has_mass) return pfe_fail(ctx, PFE_E_STATE, "chain_springs needs a context created with masses");
  if (nbonds < 0 || (nbonds > 0 && (!bi || !bj || !rhat || !k_bar)) || !vals_bar || !m_bar)
    return pfe_fail(ctx, PFE_E_ARG, "chain_springs: bad arguments");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
  launch_chain_springs(ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->H.as<double>(), ctx->mass.as<double>(),
                       nbonds, bi, bj, rhat, vals_bar, k_bar, m_bar, s);
  return check_launch(ctx, "chain_springs");
}

pfe_status pfe_solve_batch(pfe_ctx **ctxs, int32_t nsamples, int32_t *n_found) {
  if (!ctxs || nsamples < 0) return PFE_E_ARG;
  for (int32_t i = 0; i < nsamples; ++i)
    if (!ctxs[i]) return PFE_E_ARG;
  if (nsamples == 0) return PFE_OK;
  pfe_ctx *c0 = ctxs[0];
  for (int32_t i = 1; i < nsamples; ++i)
    if (ctxs[i]->device != c0->device) return pfe_fail(c0, PFE_E_ARG, "batch contexts must share one device");
  if (cudaSetDevice(c0->device) != cudaSuccess) return pfe_fail(c0, PFE_E_CUDA, "cudaSetDevice failed");
  std::vector<pfe_status> status(nsamples, PFE_OK);
  const int32_t nthreads = c0->p_batch_threads;
  bool all_bks = true, any_bks = false;
  for (int32_t i = 0; i < nsamples; ++i) {
    all_bks = all_bks && ctxs[i]->p_method == 1;
    any_bks = any_bks || ctxs[i]->p_method == 1;
  }
  if (any_bks && !all_bks) return pfe_fail(c0, PFE_E_ARG, "batch contexts must all select the same PFE_P_METHOD");
  if (all_bks) {
    // block Lanczos samples: every sample's solve on its own stream, the samples concurrently from
    // the host threads (their kernels overlap on the device); no shared graph
    std::vector<int32_t> nf(nsamples, 0);
    // Work buffers (several n x basis blocks) pass from a finished sample to the next sample its host
    // thread solves, so that only the solves in flight hold them and no device memory is freed while
    // other samples run (cudaFree synchronises the device).  The samples go largest first, so a later
    // sample rarely has to grow a buffer.  A sample that found no room beside the others runs again
    // afterwards, one at a time.
    auto work_bufs = [](pfe_ctx *c) {
      return std::vector<DBuf *>{&c->w_X, &c->w_Y, &c->w_W, &c->w_T0, &c->w_T1, &c->w_T2, &c->w_small, &c->w_small2,
                                 &c->w_red, &c->w_cs_work, &c->w_ckpt, &c->w_rr, &c->w_gram, &c->w_bks[0],
                                 &c->w_bks[1], &c->w_bks[2], &c->w_bks[3], &c->w_bks[4]};
    };
    std::vector<int32_t> order(nsamples);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return ctxs[x]->n > ctxs[y]->n; });
    int32_t nt = nthreads;
    if (nt <= 0) nt = (int32_t)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
    nt = std::max(1, std::min(nt, nsamples));
    std::atomic<int32_t> next{0};
    auto worker = [&]() {
      cudaSetDevice(c0->device);
      std::vector<DBuf> carry;  // the buffers of this thread's previous sample
      std::vector<DBuf> spare;  // smaller buffers the samples held before (freed when the thread ends)
      for (int32_t t = next.fetch_add(1); t < nsamples; t = next.fetch_add(1)) {
        const int32_t i = order[t];
        auto bufs = work_bufs(ctxs[i]);
        if (!carry.empty())
          for (size_t b = 0; b < bufs.size(); ++b)
            if (carry[b].bytes > bufs[b]->bytes) std::swap(*bufs[b], carry[b]);  // the sample takes the larger
        for (DBuf &b : carry)
          if (b.p) spare.push_back(b);
        carry.clear();
        status[i] = bks_solve(ctxs[i], &nf[i]);
        cudaStreamSynchronize(ctxs[i]->stream);  // its kernels are done with the buffers
        for (DBuf *b : bufs) {
          carry.push_back(*b);
          *b = DBuf{};
        }
      }
      for (DBuf &b : carry) dbuf_free(b);
      for (DBuf &b : spare) dbuf_free(b);
    };
    if (nt == 1) {
      worker();
    } else {
      std::vector<std::thread> pool;
      for (int32_t t = 0; t < nt; ++t) pool.emplace_back(worker);
      for (auto &th : pool) th.join();
    }
    for (int32_t i = 0; i < nsamples; ++i) {
      if (status[i] != PFE_E_NOMEM) continue;
      cudaGetLastError();  // the failed allocation's error state
      status[i] = bks_solve(ctxs[i], &nf[i]);
      for (DBuf *b : work_bufs(ctxs[i])) dbuf_free(*b);
    }
    pfe_status first = PFE_OK;
    for (int32_t i = 0; i < nsamples; ++i) {
      if (n_found) n_found[i] = nf[i];
      if (status[i] != PFE_OK && first == PFE_OK) first = status[i];
    }
    return first;
  }
  // the work buffers of a subspace-iteration solve (the locked vectors L hold the results and stay)
  auto release_si_work = [](pfe_ctx *c) {
    cudaStreamSynchronize(c->stream);
    for (DBuf *b : {&c->w_X, &c->w_Y, &c->w_W, &c->w_T0, &c->w_T1, &c->w_rr, &c->w_red, &c->w_gram, &c->w_small,
                    &c->w_small2, &c->w_cs_work, &c->w_f32a, &c->w_f32b, &c->w_f32c, &c->w_f32d, &c->w_f32e,
                    &c->w_defect, &c->w_tau})
      dbuf_free(*b);
  };
  // set-up of every sample (filter design, width, buffers, start block); a sample that failed gives
  // back what it had reserved
  for_each_sample(c0->device, nsamples, nthreads, [&](int32_t i) { status[i] = solve_setup(ctxs[i]); });
  for (int32_t i = 0; i < nsamples; ++i)
    if (status[i] != PFE_OK) {
      release_si_work(ctxs[i]);
      dbuf_free(ctxs[i]->L);  // no results yet
    }
  cudaGetLastError();  // a failed allocation's error state
  BatchPlan plan;
  pfe_status bst = batch_plan_init(c0, ctxs, nsamples, status, &plan);
  if (bst != PFE_OK) {
    batch_plan_free(&plan);
    return bst;
  }
  for (int32_t i = 0; i < nsamples; ++i) ctxs[i]->solve.timed_filter = false;
  double t_batch_filter = 0.0;
  int64_t batch_replays = 0;
  for (;;) {
    bool any = false;
    for (int32_t i = 0; i < nsamples; ++i)
      if (status[i] == PFE_OK && !ctxs[i]->solve.done) any = true;
    if (!any) break;
    // 1. filter: one batched replay for the FP64 samples, the single-context path for FP32 ones
    for_each_sample(c0->device, nsamples, nthreads, [&](int32_t i) {
      SolveState &st = ctxs[i]->solve;
      if (status[i] != PFE_OK || st.done || st.use64) return;
      status[i] = solve_filter(ctxs[i]);
    });
    float ms = 0.f;
    bst = batch_filter(c0, ctxs, nsamples, status, &plan, &ms);
    if (bst != PFE_OK) {
      batch_plan_free(&plan);
      return bst;
    }
    t_batch_filter += ms * 1e-3;
    ++batch_replays;
    // 2. everything after the filter, per sample (its own stream waits for the batched filter)
    for_each_sample(c0->device, nsamples, nthreads, [&](int32_t i) {
      SolveState &st = ctxs[i]->solve;
      if (status[i] != PFE_OK || st.done) return;
      cudaStreamWaitEvent(ctxs[i]->stream, plan.done_ev, 0);
      status[i] = solve_after_filter(ctxs[i]);
    });
  }
  batch_plan_free(&plan);
  pfe_status first = PFE_OK;
  for (int32_t i = 0; i < nsamples; ++i) {
    int32_t nf = 0;
    pfe_status fs = (status[i] == PFE_OK) ? solve_finish(ctxs[i], &nf) : status[i];
    ctxs[i]->stats.seconds_filter = t_batch_filter;  // shared by the whole batch
    ctxs[i]->stats.batch_replays = batch_replays;
    if (n_found) n_found[i] = (status[i] == PFE_OK) ? nf : 0;
    status[i] = fs;
  }
  // the batch is over: every sample gives back its work buffers; the samples that found no room
  // beside the others are solved again, one at a time (pfe_solve), each releasing its buffers after
  for (int32_t i = 0; i < nsamples; ++i) release_si_work(ctxs[i]);
  for (int32_t i = 0; i < nsamples; ++i) {
    if (status[i] != PFE_E_NOMEM) continue;
    cudaGetLastError();
    int32_t nf = 0;
    status[i] = pfe_solve(ctxs[i], &nf);
    if (n_found) n_found[i] = (status[i] == PFE_OK || status[i] == PFE_E_CAPACITY) ? nf : 0;
    release_si_work(ctxs[i]);
  }
  for (int32_t i = 0; i < nsamples; ++i)
    if (status[i] != PFE_OK && first == PFE_OK) first = status[i];
  return first;
}

}  // extern "C"
