// Thick-restart block Lanczos on the filter operator Op = p(Ht) (the block Krylov-Schur solver the
// paper runs in production, Sec. 2.5 and Sec. 3), followed by Rayleigh-Ritz with H on the converged
// wanted Op-eigenvectors ("the correct eigenvalue-eigenvector relations can be found by a
// Rayleigh-Ritz procedure applied to H", Sec. 2.5).
//
// Basis V (orthonormal, row-major n x ldv) and OV = Op V for its first nv columns:
//   expand:  OV_j = Op V_j (fused filter, bs columns); W = OV_j - V (V^T OV_j), twice (DMMA);
//            V_{j+1} = CholQR2(W), twice against V;
//   restart: T = V^T OV (DMMA Gram), T = S Theta S^T (cuSOLVER); the `keep` largest Ritz pairs
//            Y = V S, OY = OV S become the new basis; the last block V_{j+1} (orthogonal to all of
//            V) continues the Krylov sequence;
//   stop:    every Ritz pair with theta >= theta_cut has ||OY - theta Y|| <= tol_op max|theta|,
//            at least one block of Ritz values lies below theta_cut, and the number of wanted
//            pairs did not change since the previous restart.
// theta_cut = sqrt(r) min(p(xi), p(eta)): below the filter's value at the interval edges and
// above its value r min(p(xi), p(eta)) outside the margins (eq. (thresh)).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pfe_internal.h"

using namespace pfe;

namespace {

#define BKS_RESERVE(T, ptr, buf, count)                                                     \
  T *ptr = nullptr;                                                                         \
  {                                                                                         \
    cudaError_t e__ = dbuf_reserve((buf), (size_t)(count) * sizeof(T));                     \
    if (e__ != cudaSuccess)                                                                 \
      return pfe_fail(ctx, PFE_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e__)); \
    ptr = (buf).as<T>();                                                                    \
  }

pfe_status last_error(pfe_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return PFE_OK;
}

// W (n x k, ld ldw) -= V (n x nv, ld ldv) (V^T W), twice (classical Gram-Schmidt with reorthogonalisation)
pfe_status cgs2(pfe_ctx *ctx, const double *V, int64_t ldv, int32_t nv, double *W, int64_t ldw, int32_t k,
                double *h, double *gw) {
  if (nv <= 0 || k <= 0) return PFE_OK;
  for (int pass = 0; pass < 2; ++pass) {
    launch_gram(ctx->n, nv, k, V, ldv, W, ldw, 1.0, 0.0, h, nv, false, gw, ctx->stream);
    launch_update(ctx->n, k, nv, V, ldv, h, nv, -1.0, 1.0, W, ldw, ctx->stream);
  }
  return last_error(ctx, "block reorthogonalisation");
}

}  // namespace

pfe_status bks_solve(pfe_ctx *ctx, int32_t *n_found) {
  const double t_start = solver_now();
  if (ctx->p_precision != 0) return pfe_fail(ctx, PFE_E_ARG, "the block Lanczos method runs in FP64 only");
  if (!ctx->has_interval) return pfe_fail(ctx, PFE_E_STATE, "no interval set (pfe_set_interval)");
  ctx->has_result = false;
  ctx->n_found = 0;
  ctx->stats = pfe_stats{};
  PFE_TRY(solver_ensure_filter(ctx));
  PFE_TRY(solver_ensure_hs(ctx, false));
  const int64_t n = ctx->n;
  const int32_t bs = (int32_t)std::min<int64_t>(ctx->p_block, n / 4 > 0 ? n / 4 : 1);
  double window_est = 0.0;
  PFE_TRY(solver_count(ctx));
  PFE_TRY(solver_window(ctx, &window_est));
  const int32_t nev = (int32_t)std::ceil(1.1 * std::max(window_est, ctx->count_est)) + bs;
  int32_t maxbasis = (int32_t)(std::ceil(ctx->p_basis_factor * nev / bs) * bs);
  maxbasis = std::max(maxbasis, 3 * bs);
  maxbasis = (int32_t)std::min<int64_t>(maxbasis, (n - bs) / bs * bs);
  if (maxbasis < 3 * bs) return pfe_fail(ctx, PFE_E_ARG, "matrix too small for the block size");
  const int32_t keep_min = std::min(nev, maxbasis - 2 * bs);
  const int64_t ldv = (maxbasis + bs + 3) / 4 * 4, ldb = (bs + 3) / 4 * 4;
  cudaStream_t s = ctx->stream;
  // theta_cut from the filter's values at the interval edges
  const double pe = std::min(chebyshev_value(ctx->coef, ctx->m, ctx->xi), chebyshev_value(ctx->coef, ctx->m, ctx->eta));
  const double theta_cut = std::sqrt(ctx->p_rate) * pe;
  // buffers: V, OV, Y, OY, Z (n x ldv); block buffers; small matrices
  BKS_RESERVE(double, V, ctx->w_bks[0], (size_t)n * ldv);
  BKS_RESERVE(double, OV, ctx->w_bks[1], (size_t)n * ldv);
  BKS_RESERVE(double, Y, ctx->w_bks[2], (size_t)n * ldv);
  BKS_RESERVE(double, OY, ctx->w_bks[3], (size_t)n * ldv);
  BKS_RESERVE(double, Z, ctx->L, (size_t)n * ldv);  // final eigenvectors live in ctx->L
  BKS_RESERVE(double, Xb, ctx->w_X, (size_t)n * ldb * 5);
  double *Yb = Xb + (size_t)n * ldb, *T0b = Yb + (size_t)n * ldb, *T1b = T0b + (size_t)n * ldb,
         *Wb = T1b + (size_t)n * ldb;
  BKS_RESERVE(double, T, ctx->w_rr, (size_t)maxbasis * maxbasis + 3 * (size_t)maxbasis + 8);
  // evals: Ritz values; dres: the kept Ritz values (residual input); rout: residual norms squared
  double *evals = T + (size_t)maxbasis * maxbasis, *dres = evals + maxbasis, *rout = dres + maxbasis;
  BKS_RESERVE(double, h, ctx->w_small2, (size_t)(maxbasis + bs) * std::max(bs, 1) + 8);
  BKS_RESERVE(double, gw, ctx->w_gram,
              std::max(gram_work(n, maxbasis + bs, bs, false), gram_work(n, maxbasis, maxbasis, false)));
  BKS_RESERVE(double, red, ctx->w_red, colreduce_work(n, maxbasis) + 8);
  BKS_RESERVE(int, info, ctx->w_info, 4);
  for (double *p : {V, OV, Y, OY, Z}) launch_zero<double>(p, n * ldv, s);
  launch_zero<double>(Xb, n * ldb * 5, s);
  const double tol = ctx->p_tol;
  const int max_restarts = std::max(ctx->p_max_iters, 1);
  double tol_op = 1e-10, t_filter = 0.0, t_orth = 0.0, t_rr = 0.0;
  int64_t matvecs = 0, f_launch = 0, f_cols = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](double &acc) {
    float ms = 0;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    acc += ms * 1e-3;
    cudaEventRecord(e0, s);
  };
  cudaEventRecord(e0, s);
  // start block: Philox normals of stream 0, orthonormalised
  launch_fill_normal<double>(ctx->p_seed, 0u, n, bs, 0, Wb, ldb, s);
  {
    double *res = nullptr;
    PFE_TRY(solver_cholqr2(ctx, Wb, T0b, bs, ldb, &res));
    launch_axpby<double>(n, bs, 1.0, res, ldb, 0.0, V, ldv, s);
  }
  int32_t nv = 0, restarts = 0, prev_nwant = -1, nf = 0;
  pfe_status result = PFE_E_NOCONV;
  std::vector<double> hev, hres;
  std::vector<int32_t> sel_cols;
  std::vector<double> sel_lam, sel_res;
  for (;;) {
    // ---- expand the basis while another block fits
    while (nv + bs <= maxbasis) {
      launch_axpby<double>(n, bs, 1.0, V + nv, ldv, 0.0, Xb, ldb, s);
      cudaEventRecord(e0, s);
      PFE_TRY(solver_filter64(ctx, bs, ldb, Xb, Yb, T0b, T1b));
      timed(t_filter);
      matvecs += (int64_t)bs * ctx->m;
      f_launch += std::max(ctx->m, 1);
      f_cols += (int64_t)bs * std::max(ctx->m, 1);
      launch_axpby<double>(n, bs, 1.0, Yb, ldb, 0.0, OV + nv, ldv, s);
      launch_axpby<double>(n, bs, 1.0, Yb, ldb, 0.0, Wb, ldb, s);
      double *res = nullptr;
      for (int rep = 0; rep < 2; ++rep) {
        PFE_TRY(cgs2(ctx, V, ldv, nv + bs, Wb, ldb, bs, h, gw));
        PFE_TRY(solver_cholqr2(ctx, Wb, T0b, bs, ldb, &res));
        if (res != Wb) launch_axpby<double>(n, bs, 1.0, res, ldb, 0.0, Wb, ldb, s);
      }
      launch_axpby<double>(n, bs, 1.0, Wb, ldb, 0.0, V + nv + bs, ldv, s);
      PFE_TRY(last_error(ctx, "expansion"));
      nv += bs;
      timed(t_orth);
    }
    // ---- Rayleigh-Ritz of Op on span(V): T = V^T OV, eigen-decomposition
    launch_gram(n, nv, nv, V, ldv, OV, ldv, 1.0, 0.0, T, nv, false, gw, s);
    int lw = 0;
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, nv,
                                                    T, nv, evals, &lw));
    BKS_RESERVE(double, work, ctx->w_cs_work, (size_t)std::max(lw, 1));
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, nv, T, nv,
                                         evals, work, lw, info));
    hev.resize(nv);
    int hinfo = 0;
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hev.data(), evals, sizeof(double) * nv, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hinfo != 0) return pfe_fail(ctx, PFE_E_CUDA, "cusolverDnDsyevd did not converge");
    // wanted: Ritz values >= theta_cut (they are the last ones: ascending order)
    int32_t nwant = 0;
    for (int32_t i = 0; i < nv; ++i)
      if (hev[i] >= theta_cut) ++nwant;
    int32_t keep = std::max(nwant + bs, keep_min);
    keep = std::min(keep, nv - bs);
    keep = std::max(keep, nwant);
    // the kept Ritz pairs: Y = V S[:, nv-keep:], OY = OV S[:, nv-keep:]
    launch_update(n, keep, nv, V, ldv, T + (size_t)(nv - keep) * nv, nv, 1.0, 0.0, Y, ldv, s);
    launch_update(n, keep, nv, OV, ldv, T + (size_t)(nv - keep) * nv, nv, 1.0, 0.0, OY, ldv, s);
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(dres, evals + (nv - keep), sizeof(double) * keep, cudaMemcpyDeviceToDevice, s));
    launch_col_resid2(n, keep, OY, Y, ldv, dres, rout, red, s);
    hres.resize(keep);
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hres.data(), rout, sizeof(double) * keep, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    PFE_TRY(last_error(ctx, "Ritz pairs"));
    timed(t_rr);
    double thmax = 0.0;
    for (int32_t i = 0; i < nv; ++i) thmax = std::max(thmax, std::fabs(hev[i]));
    int32_t nconv = 0;
    for (int32_t i = keep - nwant; i < keep; ++i)
      if (std::sqrt(std::max(hres[i], 0.0)) <= tol_op * thmax) ++nconv;
    if (nwant > nv - bs) {  // the wanted Ritz values fill the basis: completeness cannot be shown
      result = PFE_E_CAPACITY;
      break;
    }
    const bool done = nwant == nconv && nwant == prev_nwant;
    prev_nwant = nwant;
    if (done) {
      // ---- Rayleigh-Ritz with H on the wanted Op-eigenvectors Yw = Y[:, keep - nwant : keep]
      const double *Yw = Y + (keep - nwant);
      const int32_t k = nwant;
      sel_cols.clear();
      sel_lam.clear();
      sel_res.clear();
      bool bad = false;
      if (k > 0) {
        launch_bsr_step<double>(Bsr<double>{ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->H.as<double>()},
                                MODE_SPMM, k, ldv, Yw, nullptr, OV, nullptr, 1.0, 0.0, 0.0, 0.0, s);
        matvecs += k;
        launch_gram(n, k, k, Yw, ldv, OV, ldv, 1.0, 0.0, T, k, false, gw, s);
        PFE_SOLVER_TRY(ctx, cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k,
                                                        T, k, evals, &lw));
        BKS_RESERVE(double, work2, ctx->w_cs_work, (size_t)std::max(lw, 1));
        PFE_SOLVER_TRY(ctx, cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k, T, k,
                                             evals, work2, lw, info));
        launch_update(n, k, k, Yw, ldv, T, k, 1.0, 0.0, Z, ldv, s);  // U = Yw Q
        launch_bsr_step<double>(Bsr<double>{ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->H.as<double>()},
                                MODE_SPMM, k, ldv, Z, nullptr, OV, nullptr, 1.0, 0.0, 0.0, 0.0, s);
        matvecs += k;
        launch_col_resid2(n, k, OV, Z, ldv, evals, rout, red, s);
        std::vector<double> lam(k), r2(k);
        PFE_CUDA_TRY(ctx, cudaMemcpyAsync(lam.data(), evals, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
        PFE_CUDA_TRY(ctx, cudaMemcpyAsync(r2.data(), rout, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
        PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
        PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (hinfo != 0) return pfe_fail(ctx, PFE_E_CUDA, "cusolverDnDsyevd did not converge");
        PFE_TRY(last_error(ctx, "final Rayleigh-Ritz"));
        for (int32_t j = 0; j < k; ++j) {
          if (lam[j] < ctx->a || lam[j] > ctx->b) continue;
          const double rel = std::sqrt(std::max(r2[j], 0.0)) / ctx->lmax;
          if (rel > tol) bad = true;
          sel_cols.push_back(j);
          sel_lam.push_back(lam[j]);
          sel_res.push_back(rel * ctx->lmax);
        }
      }
      timed(t_rr);
      if (!bad) {
        result = (nwant >= maxbasis - bs) ? PFE_E_CAPACITY : PFE_OK;
        nf = (int32_t)sel_cols.size();
        break;
      }
      if (tol_op < 1e-15) {
        nf = (int32_t)sel_cols.size();
        result = PFE_E_NOCONV;
        break;
      }
      tol_op *= 1e-2;  // the Op-residuals were not yet small enough for the H-residuals
      // OV was overwritten by the final Rayleigh-Ritz: OY still holds Op Y for the restart below
    }
    if (++restarts > max_restarts) {
      result = PFE_E_NOCONV;
      break;
    }
    // ---- thick restart: the kept Ritz pairs, then the continuation block V[:, nv : nv + bs]
    launch_axpby<double>(n, bs, 1.0, V + nv, ldv, 0.0, Wb, ldb, s);
    launch_axpby<double>(n, keep, 1.0, Y, ldv, 0.0, V, ldv, s);
    launch_axpby<double>(n, keep, 1.0, OY, ldv, 0.0, OV, ldv, s);
    {
      double *res = nullptr;
      PFE_TRY(cgs2(ctx, V, ldv, keep, Wb, ldb, bs, h, gw));
      PFE_TRY(solver_cholqr2(ctx, Wb, T0b, bs, ldb, &res));
      launch_axpby<double>(n, bs, 1.0, res, ldb, 0.0, V + keep, ldv, s);
    }
    PFE_TRY(last_error(ctx, "restart"));
    nv = keep;
    timed(t_orth);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // results: columns of Z (= ctx->L) in ascending eigenvalue order (syevd returns ascending)
  ctx->ldq = ldv;
  ctx->result_cols = sel_cols;
  ctx->result_lam = sel_lam;
  ctx->result_res = sel_res;
  ctx->n_found = nf;
  ctx->has_result = result == PFE_OK || result == PFE_E_CAPACITY || nf > 0;
  pfe_stats &o = ctx->stats;
  o.iterations = restarts;
  o.restarts = restarts;
  o.basis = maxbasis;
  o.width = bs;
  o.degree = ctx->m;
  o.n_found = nf;
  o.matvecs = matvecs;
  o.lambda_max = ctx->lmax;
  o.count_estimate = ctx->count_est;
  o.window_estimate = window_est;
  o.seconds_filter = t_filter;
  o.seconds_orth = t_orth;
  o.seconds_rr = t_rr;
  double mr = 0.0;
  for (double r : sel_res) mr = std::max(mr, r / ctx->lmax);
  o.max_residual = mr;
  o.fp64_sweeps = 0;
  o.status = (int32_t)result;
  o.kernel_launches = launch_count() - ctx->launch_base;
  o.filter_launches = f_launch;
  o.filter_col_steps = f_cols;
  o.seconds_total = solver_now() - t_start;
  if (n_found) *n_found = nf;
  if (result == PFE_E_CAPACITY) return pfe_fail(ctx, result, "the wanted Ritz values fill the basis: raise BASIS_FACTOR");
  if (result == PFE_E_NOCONV) return pfe_fail(ctx, result, "restart limit reached");
  return PFE_OK;
}
