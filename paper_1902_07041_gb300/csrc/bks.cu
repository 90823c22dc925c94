// Thick-restart block Lanczos on the filter operator Op = p(Ht) (the block Krylov-Schur solver the
// paper runs in production, Sec. 2.5 and Sec. 3), followed by Rayleigh-Ritz with H on the wanted
// Op-eigenvectors: the eigenvectors of Op are those of H, and a Rayleigh-Ritz step with H recovers
// the eigenvalues (Sec. 2.5).
//
// Basis V (orthonormal, row-major n x ldv) with the Krylov-Schur relation
//     Op V[:, 0:nv] = V[:, 0:nv] T + V[:, nv:nv+bs] B E^T,
// T (nv x nv, symmetric, its upper triangle kept on the device) and B = V[:, nv:nv+bs]^T Op V_last
// (bs x bs; E^T selects the last block of columns).
//   expand:  Yb = Op V_j (fused filter, bs columns); the first Gram-Schmidt pass h = V^T Yb is the
//            new column block of T, W = Yb - V h, a second pass against V (DMMA), then
//            V_{j+1} = CholQR2(W); a numerically rank-deficient W (shifted CholQR) is projected and
//            factored once more;
//   Ritz:    T = S Theta S^T (cuSOLVER); the residual of Ritz pair i is ||B s_i[nv-bs:nv]||, from
//            bs x nv numbers on the host: no n-length work;
//   restart: the `keep` largest Ritz pairs Y = V S[:, nv-keep:] become the new basis with
//            T = diag(theta); the block V[:, nv:nv+bs] (orthogonal to all of V) continues the
//            Krylov sequence, and its first expansion fills the coupling column block of T;
//   stop:    every Ritz pair with theta >= theta_cut has residual <= tol_op max|theta|, at least one
//            block of Ritz values lies below theta_cut, and the number of wanted pairs did not
//            change since the previous restart.
// theta_cut, piecewise quadratic filter: sqrt(r) min(p(xi), p(eta)), below the filter's value at the
// interval edges and above its value r min(p(xi), p(eta)) outside the margins (eq. (thresh)).  Dirac
// filter (eq. (cheby-delta.1), centred so that rho(xi) = rho(eta) = tau, above tau inside the
// interval): DIRAC_CUT tau, 0.9 tau by default.
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

// W (n x k, ld ldw) -= V (n x nv, ld ldv) (V^T W), `passes` times; h (col-major nv x k, ld nv)
// receives the last V^T W
void project(pfe_ctx *ctx, const double *V, int64_t ldv, int32_t nv, double *W, int64_t ldw, int32_t k, double *h,
             double *gw, int passes) {
  if (nv <= 0 || k <= 0) return;
  for (int pass = 0; pass < passes; ++pass) {
    launch_gram(ctx->n, nv, k, V, ldv, W, ldw, 1.0, 0.0, h, nv, false, gw, ctx->stream);
    launch_update(ctx->n, k, nv, V, ldv, h, nv, -1.0, 1.0, W, ldw, ctx->stream);
  }
}

// Orthonormalise W (n x bs, ld ldb) against V[:, 0:nv] and within itself: `first_passes` projection
// passes and CholQR2, repeated with two passes when the block was numerically rank deficient (a
// shifted factorisation).  The result is left in W.
pfe_status orthonormalise_block(pfe_ctx *ctx, const double *V, int64_t ldv, int32_t nv, double *W, double *tmp,
                                int64_t ldb, int32_t bs, double *h, double *gw, int first_passes) {
  cudaStream_t s = ctx->stream;
  for (int rep = 0; rep < 2; ++rep) {
    project(ctx, V, ldv, nv, W, ldb, bs, h, gw, rep == 0 ? first_passes : 2);
    double *res = nullptr;
    bool shifted = false;
    PFE_TRY(solver_cholqr2(ctx, W, tmp, bs, ldb, &res, &shifted));
    if (res != W) launch_axpby<double>(ctx->n, bs, 1.0, res, ldb, 0.0, W, ldb, s);
    if (!shifted) break;
  }
  return last_error(ctx, "block orthonormalisation");
}

}  // namespace

pfe_status bks_solve(pfe_ctx *ctx, int32_t *n_found) {
  const double t_start = solver_now();
  if (ctx->p_precision != 0) return pfe_fail(ctx, PFE_E_ARG, "the block Lanczos method runs in FP64 only");
  if (!ctx->has_interval) return pfe_fail(ctx, PFE_E_STATE, "no interval set (pfe_set_interval)");
  ctx->has_result = false;
  ctx->n_found = 0;
  ctx->stats = pfe_stats{};
  ctx->shift_count = 0;
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
  const int64_t ldv = (maxbasis + bs + 3) / 4 * 4, ldb = (bs + 3) / 4 * 4, ldT = maxbasis;
  cudaStream_t s = ctx->stream;
  // wanted Ritz values of Op: piecewise quadratic filter, theta >= sqrt(r) min(p(xi), p(eta)); Dirac
  // filter, theta >= DIRAC_CUT x tau with tau = rho(xi) = rho(eta)
  const double pe = std::min(chebyshev_value(ctx->coef, ctx->m, ctx->xi), chebyshev_value(ctx->coef, ctx->m, ctx->eta));
  const double theta_cut = (ctx->p_filter == 1) ? ctx->p_dirac_cut * ctx->dirac_tau : std::sqrt(ctx->rate_of()) * pe;
  // n x ldv buffers: V (basis), Vn (next basis, or the wanted Ritz vectors), HW (products with H),
  // Z = ctx->L (the returned eigenvectors)
  BKS_RESERVE(double, V, ctx->w_bks[0], (size_t)n * ldv);
  BKS_RESERVE(double, Vn, ctx->w_bks[1], (size_t)n * ldv);
  BKS_RESERVE(double, HW, ctx->w_bks[2], (size_t)n * ldv);
  BKS_RESERVE(double, Z, ctx->L, (size_t)n * ldv);
  for (int i = 3; i < 5; ++i) dbuf_free(ctx->w_bks[i]);
  BKS_RESERVE(double, Xb, ctx->w_X, (size_t)n * ldb * 5);
  double *Yb = Xb + (size_t)n * ldb, *T0b = Yb + (size_t)n * ldb, *T1b = T0b + (size_t)n * ldb,
         *Wb = T1b + (size_t)n * ldb;
  // small: Tm (maxbasis x maxbasis col-major: the upper triangle of T), A (Ritz vectors S, ld nv),
  // evals, fin_lam / fin_r2 (the final step's eigenvalues and squared residuals), Bm (bs x bs)
  const size_t mb = (size_t)maxbasis;
  BKS_RESERVE(double, Tm, ctx->w_rr, 2 * mb * mb + 3 * mb + (size_t)bs * bs + 8);
  double *A = Tm + mb * mb, *evals = A + mb * mb, *fin_lam = evals + mb, *fin_r2 = fin_lam + mb, *Bm = fin_r2 + mb;
  BKS_RESERVE(double, h, ctx->w_small2, (mb + bs) * (size_t)std::max(bs, 1) + 8);
  BKS_RESERVE(double, gw, ctx->w_gram,
              std::max({gram_work(n, maxbasis + bs, bs, false), gram_work(n, maxbasis, maxbasis, false),
                        gram_work(n, bs, bs, true)}));  // CholQR2 reuses this buffer: it must not grow
  BKS_RESERVE(double, red, ctx->w_red, colreduce_work(n, maxbasis) + 8);
  BKS_RESERVE(int, info, ctx->w_info, 4);
  launch_zero<double>(V, n * ldv, s);
  launch_zero<double>(Xb, n * ldb * 5, s);
  launch_zero<double>(Tm, (int64_t)(mb * mb), s);
  const double tol = ctx->p_tol;
  const int max_restarts = std::max(ctx->p_max_iters, 1);
  double tol_op = 1e-10, t_filter = 0.0, t_orth = 0.0, t_rr = 0.0;
  int64_t matvecs = 0, f_launch = 0, f_cols = 0;
  struct Events {  // destroyed on every return path
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Events() {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
    }
    ~Events() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    }
  } events;
  cudaEvent_t e0 = events.e0, e1 = events.e1;
  auto timed = [&](double &acc) {
    float ms = 0;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    acc += ms * 1e-3;
    cudaEventRecord(e0, s);
  };
  const Bsr<double> Hb{ctx->N, ctx->rp.as<int32_t>(), ctx->ci.as<int32_t>(), ctx->H.as<double>()};
  cudaEventRecord(e0, s);
  // start block: Philox normals of stream 0, orthonormalised
  launch_fill_normal<double>(ctx->p_seed, 0u, n, bs, 0, Wb, ldb, s);
  PFE_TRY(orthonormalise_block(ctx, V, ldv, 0, Wb, T0b, ldb, bs, h, gw, 2));
  launch_axpby<double>(n, bs, 1.0, Wb, ldb, 0.0, V, ldv, s);
  int32_t nv = 0, restarts = 0, prev_nwant = -1, nf = 0;
  pfe_status result = PFE_E_NOCONV;
  std::vector<double> hev, hS, hB, hres, hkeep;
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
      launch_axpby<double>(n, bs, 1.0, Yb, ldb, 0.0, Wb, ldb, s);
      // first pass: T[0:nv+bs, nv:nv+bs] = V^T Op V_j, then W -= V T[0:nv+bs, nv:nv+bs]
      double *Tcol = Tm + (size_t)nv * ldT;
      launch_gram(n, nv + bs, bs, V, ldv, Wb, ldb, 1.0, 0.0, Tcol, ldT, false, gw, s);
      launch_update(n, bs, nv + bs, V, ldv, Tcol, ldT, -1.0, 1.0, Wb, ldb, s);
      PFE_TRY(orthonormalise_block(ctx, V, ldv, nv + bs, Wb, T0b, ldb, bs, h, gw, 1));
      launch_axpby<double>(n, bs, 1.0, Wb, ldb, 0.0, V + nv + bs, ldv, s);
      nv += bs;
      timed(t_orth);
    }
    // ---- Ritz pairs of T; B = V_new^T Op V_last (Yb holds Op V_last)
    launch_gram(n, bs, bs, V + nv, ldv, Yb, ldb, 1.0, 0.0, Bm, bs, false, gw, s);
    PFE_CUDA_TRY(ctx, cudaMemcpy2DAsync(A, sizeof(double) * nv, Tm, sizeof(double) * ldT, sizeof(double) * nv, nv,
                                        cudaMemcpyDeviceToDevice, s));
    int lw = 0;
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, nv,
                                                    A, nv, evals, &lw));
    BKS_RESERVE(double, work, ctx->w_cs_work, (size_t)std::max(lw, 1));
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, nv, A, nv,
                                         evals, work, lw, info));
    hev.resize(nv);
    hS.resize((size_t)bs * nv);
    hB.resize((size_t)bs * bs);
    int hinfo = 0;
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hev.data(), evals, sizeof(double) * nv, cudaMemcpyDeviceToHost, s));
    // the last bs rows of every Ritz vector s_i (column i of A, ld nv)
    PFE_CUDA_TRY(ctx, cudaMemcpy2DAsync(hS.data(), sizeof(double) * bs, A + (nv - bs), sizeof(double) * nv,
                                        sizeof(double) * bs, nv, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hB.data(), Bm, sizeof(double) * bs * bs, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    PFE_TRY(last_error(ctx, "Ritz pairs"));
    if (hinfo != 0) return pfe_fail(ctx, PFE_E_CUDA, "cusolverDnDsyevd did not converge");
    timed(t_rr);
    // residuals ||B s_i,last|| (B col-major bs x bs)
    hres.assign(nv, 0.0);
    for (int32_t i = 0; i < nv; ++i) {
      const double *sl = hS.data() + (size_t)i * bs;
      double acc = 0.0;
      for (int32_t r = 0; r < bs; ++r) {
        double v = 0.0;
        for (int32_t c = 0; c < bs; ++c) v += hB[(size_t)c * bs + r] * sl[c];
        acc += v * v;
      }
      hres[i] = std::sqrt(acc);
    }
    // wanted: Ritz values >= theta_cut (the last ones: ascending order)
    int32_t nwant = 0;
    double thmax = 0.0;
    for (int32_t i = 0; i < nv; ++i) {
      if (hev[i] >= theta_cut) ++nwant;
      thmax = std::max(thmax, std::fabs(hev[i]));
    }
    int32_t keep = std::max(nwant + bs, keep_min);
    keep = std::min(keep, nv - bs);
    keep = std::max(keep, nwant);
    int32_t nconv = 0;
    for (int32_t i = nv - nwant; i < nv; ++i)
      if (hres[i] <= tol_op * thmax) ++nconv;
    if (nwant > nv - bs) {  // the wanted Ritz values fill the basis: completeness cannot be shown
      result = PFE_E_CAPACITY;
      break;
    }
    const bool done = nwant == nconv && nwant == prev_nwant;
    prev_nwant = nwant;
    if (done) {
      // ---- Rayleigh-Ritz with H on the wanted Op-eigenvectors Yw = V S[:, nv - nwant : nv] (in Vn)
      const int32_t k = nwant;
      sel_cols.clear();
      sel_lam.clear();
      sel_res.clear();
      bool bad = false;
      if (k > 0) {
        launch_update(n, k, nv, V, ldv, A + (size_t)(nv - k) * nv, nv, 1.0, 0.0, Vn, ldv, s);
        launch_bsr_step<double>(Hb, MODE_SPMM, k, ldv, Vn, nullptr, HW, nullptr, 1.0, 0.0, 0.0, 0.0, s);
        matvecs += k;
        {
          BKS_RESERVE(double, gw2, ctx->w_gram, std::max(gram_work(n, k, k, true), gram_work(n, k, k, false)));
          gw = gw2;  // the buffer may have grown
        }
        double *G = Tm;  // T is rebuilt by the restart below if the iteration has to continue
        launch_gram(n, k, k, Vn, ldv, HW, ldv, 1.0, 0.0, G, k, true, gw, s);  // Yw^T H Yw: symmetric
        PFE_SOLVER_TRY(ctx, cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k,
                                                        G, k, fin_lam, &lw));
        BKS_RESERVE(double, work2, ctx->w_cs_work, (size_t)std::max(lw, 1));
        PFE_SOLVER_TRY(ctx, cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, k, G, k,
                                             fin_lam, work2, lw, info));
        launch_update(n, k, k, Vn, ldv, G, k, 1.0, 0.0, Z, ldv, s);  // U = Yw Q
        launch_bsr_step<double>(Hb, MODE_SPMM, k, ldv, Z, nullptr, HW, nullptr, 1.0, 0.0, 0.0, 0.0, s);
        matvecs += k;
        launch_col_resid2(n, k, HW, Z, ldv, fin_lam, fin_r2, red, s);
        std::vector<double> lam(k), r2(k);
        PFE_CUDA_TRY(ctx, cudaMemcpyAsync(lam.data(), fin_lam, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
        PFE_CUDA_TRY(ctx, cudaMemcpyAsync(r2.data(), fin_r2, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
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
        timed(t_rr);
      }
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
    }
    if (++restarts > max_restarts) {
      result = PFE_E_NOCONV;
      break;
    }
    // ---- thick restart: [V S[:, nv-keep:nv] | V[:, nv:nv+bs]] becomes the basis, T = diag(theta_kept)
    launch_update(n, keep, nv, V, ldv, A + (size_t)(nv - keep) * nv, nv, 1.0, 0.0, Vn, ldv, s);
    launch_axpby<double>(n, bs, 1.0, V + nv, ldv, 0.0, Wb, ldb, s);
    std::swap(V, Vn);
    PFE_TRY(orthonormalise_block(ctx, V, ldv, keep, Wb, T0b, ldb, bs, h, gw, 2));
    launch_axpby<double>(n, bs, 1.0, Wb, ldb, 0.0, V + keep, ldv, s);
    launch_zero<double>(Tm, (int64_t)(mb * mb), s);
    hkeep.assign(hev.end() - keep, hev.end());
    PFE_CUDA_TRY(ctx, cudaMemcpy2DAsync(Tm, sizeof(double) * (ldT + 1), hkeep.data(), sizeof(double), sizeof(double),
                                        keep, cudaMemcpyHostToDevice, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // hkeep must outlive its copy
    PFE_TRY(last_error(ctx, "restart"));
    nv = keep;
    timed(t_orth);
  }
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
  o.cholqr_shifts = ctx->shift_count;
  o.status = (int32_t)result;
  o.kernel_launches = launch_count() - ctx->launch_base;
  o.filter_launches = f_launch;
  o.filter_col_steps = f_cols;
  o.filter_shape_f64 = f_cols > 0 ? step_last_variant(0) : -1;
  o.filter_shape_f32 = -1;
  o.seconds_total = solver_now() - t_start;
  if (n_found) *n_found = nf;
  if (result == PFE_E_CAPACITY) return pfe_fail(ctx, result, "the wanted Ritz values fill the basis: raise BASIS_FACTOR");
  if (result == PFE_E_NOCONV) return pfe_fail(ctx, result, "restart limit reached");
  return PFE_OK;
}
