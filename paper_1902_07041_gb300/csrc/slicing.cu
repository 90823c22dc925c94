// Spectrum slicing: [a, b] split into sub-intervals that each hold a reasonable number of
// eigenvalues (Sec. 2.6: when the subspace would grow too large; Sec. 5: for memory), each solved by
// the selected method, the eigenpairs merged.
//
// Edges.  The cumulative eigenvalue count inside [a, b] comes from the stochastic estimator of
// Sec. 2.4 written with Chebyshev moments: mu_j = sum_l v_l^T T_j(Ht) v_l for M normalised Gaussian
// vectors, one recurrence of degree D, and then the count of any [x0, x1] is
// (n / M) sum_j g_j c_j(x0, x1) mu_j with the characteristic function's coefficients c_j (App. A)
// and Jackson factors g_j (a nonnegative kernel: the cumulative count is monotone).  The edges are
// where it crosses multiples of count / slices.
//
// Merge.  Slice i is solved on [e_i - delta, e_{i+1} + delta] (delta = 1e-6 lambda_max, not beyond
// [a, b]).  Near every interior edge e the pairs of both neighbours with |lambda - e| <= 2 delta are
// gathered into W; the eigenvalues of W^T W are ~2 on a direction both slices found and ~1 on one
// found once, so the directions with W^T W eigenvalue > 1/2 give an orthonormal basis of their
// joint span, and a Rayleigh-Ritz step with H on it returns each eigenpair once.  No decision
// depends on comparing two independently computed eigenvalues with the edge.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "pfe_internal.h"

using namespace pfe;

namespace {

#define SL_RESERVE(T, ptr, buf, count)                                                      \
  T *ptr = nullptr;                                                                         \
  {                                                                                         \
    cudaError_t e__ = dbuf_reserve((buf), (size_t)(count) * sizeof(T));                     \
    if (e__ != cudaSuccess)                                                                 \
      return pfe_fail(ctx, PFE_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e__)); \
    ptr = (buf).as<T>();                                                                    \
  }

pfe_status sl_error(pfe_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return PFE_OK;
}

// Chebyshev moments mu_j = sum_l v_l^T T_j(Ht) v_l, j = 0..D, of M normalised Philox vectors
// (stream 3), from the operator A = 2 Ht: t_1 = A t_0 / 2, t_{j+1} = A t_j - t_{j-1}.
pfe_status dos_moments(pfe_ctx *ctx, int32_t D, int32_t M, std::vector<double> &mu) {
  const int64_t n = ctx->n, ld = (M + 1) / 2 * 2;
  cudaStream_t s = ctx->stream;
  SL_RESERVE(double, V, ctx->w_X, (size_t)n * ld);
  SL_RESERVE(double, T0, ctx->w_Y, (size_t)n * ld);
  SL_RESERVE(double, T1, ctx->w_T0, (size_t)n * ld);
  SL_RESERVE(double, dots, ctx->w_small, (size_t)(D + 1) * M + (size_t)M + 8);
  SL_RESERVE(double, red, ctx->w_red, colreduce_work(n, M));
  launch_zero<double>(V, n * ld, s);
  launch_fill_normal<double>(ctx->p_seed, 3u, n, M, 0, V, ld, s);
  launch_col_dots<double>(n, M, V, ld, V, ld, dots, red, s);
  std::vector<double> nrm(M);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(nrm.data(), dots, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  for (auto &v : nrm) v = 1.0 / std::sqrt(v);
  double *inv = dots + (size_t)(D + 1) * M;
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(inv, nrm.data(), sizeof(double) * M, cudaMemcpyHostToDevice, s));
  launch_scale_cols<double>(n, M, V, ld, inv, s);
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // nrm must outlive its copy
  const Bsr<double> A = solver_bsr_Hs64(ctx);
  launch_col_dots<double>(n, M, V, ld, V, ld, dots, red, s);  // mu_0
  const double *tp = V;
  double *tc = T0, *spare = T1;
  if (D >= 1) {
    launch_bsr_step<double>(A, MODE_SPMM, M, ld, V, nullptr, tc, nullptr, 0.5, 0.0, 0.0, 0.0, s);
    launch_col_dots<double>(n, M, V, ld, tc, ld, dots + M, red, s);
  }
  for (int32_t j = 1; j < D; ++j) {
    double *out = (tp == V) ? spare : const_cast<double *>(tp);
    launch_bsr_step<double>(A, MODE_STEP, M, ld, tc, tp, out, nullptr, 1.0, -1.0, 0.0, 0.0, s);
    launch_col_dots<double>(n, M, V, ld, out, ld, dots + (size_t)(j + 1) * M, red, s);
    tp = tc;
    tc = out;
  }
  std::vector<double> h((size_t)(D + 1) * M);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), dots, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  PFE_TRY(sl_error(ctx, "density-of-states moments"));
  mu.assign((size_t)D + 1, 0.0);
  for (int32_t j = 0; j <= D; ++j)
    for (int32_t l = 0; l < M; ++l) mu[j] += h[(size_t)j * M + l];
  return PFE_OK;
}

// estimated count in [x0, x1] (transformed units) from the moments
double dos_count(const std::vector<double> &mu, const std::vector<double> &g, int32_t D, double x0, double x1,
                 double scale) {
  std::vector<double> c;
  chi_coefficients(std::max(x0, -1.0), std::min(x1, 1.0), D, c);
  double v = 0.0;
  for (int32_t j = 0; j <= D; ++j) v += g[j] * c[j] * mu[j];
  return scale * v;
}

struct Pair {
  double lam, res;
  int32_t slice;
  int64_t col;  // column in the accumulation buffer
};

}  // namespace

extern "C" pfe_status pfe_solve_sliced(pfe_ctx *ctx, int32_t nedges, const double *edges_in, int32_t *n_found) {
  if (!ctx) return PFE_E_ARG;
  if (!ctx->has_interval) return pfe_fail(ctx, PFE_E_STATE, "no interval set (pfe_set_interval)");
  if (nedges < 0 || (nedges > 0 && !edges_in)) return pfe_fail(ctx, PFE_E_ARG, "solve_sliced: bad edges");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  const double t_start = solver_now();
  const double a = ctx->a, b = ctx->b;
  PFE_TRY(solver_ensure_lmax(ctx));
  PFE_TRY(solver_ensure_hs(ctx, false));
  const int64_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  // ---- edges
  std::vector<double> e;  // all edges: a, interior..., b
  e.push_back(a);
  if (nedges > 0) {
    for (int32_t i = 0; i < nedges; ++i) {
      if (!(edges_in[i] > e.back() && edges_in[i] < b)) return pfe_fail(ctx, PFE_E_ARG, "solve_sliced: edges must increase inside (a, b)");
      e.push_back(edges_in[i]);
    }
  } else {
    PFE_TRY(solver_count(ctx));
    const double total = std::max(ctx->count_est, 0.0);
    const int32_t S = std::max<int32_t>(1, (int32_t)std::lround(total / std::max(ctx->p_slice_target, 1)));
    if (S > 1) {
      const double xa = (a - ctx->tc) / ctx->td, xb = (b - ctx->tc) / ctx->td;
      // resolution of the moments: about 16 Chebyshev wavelengths per slice
      const int32_t D = (int32_t)std::min(8000.0, std::max((double)ctx->p_count_degree, std::ceil(16.0 * S / (xb - xa))));
      const int32_t M = std::max(ctx->p_count_m, 1);
      std::vector<double> mu, g;
      PFE_TRY(dos_moments(ctx, D, M, mu));
      damping_factors(1, D, g);
      const double scale = (double)n / (double)M;
      const int32_t grid = 64 * S;
      std::vector<double> cum(grid + 1, 0.0);
      for (int32_t k = 1; k <= grid; ++k) cum[k] = dos_count(mu, g, D, xa, xa + (xb - xa) * k / grid, scale);
      for (int32_t k = 1; k <= grid; ++k) cum[k] = std::max(cum[k], cum[k - 1]);  // monotone
      const double tot = cum[grid];
      for (int32_t i = 1; i < S; ++i) {
        const double want = tot * i / S;
        int32_t k = 1;
        while (k < grid && cum[k] < want) ++k;
        const double f = (cum[k] > cum[k - 1]) ? (want - cum[k - 1]) / (cum[k] - cum[k - 1]) : 0.5;
        const double x = xa + (xb - xa) * (k - 1 + f) / grid;
        const double lam = ctx->tc + ctx->td * x;
        if (lam > e.back() && lam < b) e.push_back(lam);
      }
    }
  }
  e.push_back(b);
  const int32_t S = (int32_t)e.size() - 1;
  if (S == 1) return pfe_solve(ctx, n_found);
  // ---- solve every slice; gather its eigenvectors into the accumulation buffer
  const double delta = 1e-6 * ctx->lmax;
  std::vector<Pair> pairs;
  int64_t cap = 0, used = 0, ldacc = 0;
  DBuf *acc = &ctx->w_slice[0], *tmpb = &ctx->w_slice[1];
  pfe_stats sum{};
  pfe_status worst = PFE_OK;
  for (int32_t i = 0; i < S; ++i) {
    const double lo = (i == 0) ? a : std::max(a, e[i] - delta), hi = (i == S - 1) ? b : std::min(b, e[i + 1] + delta);
    ctx->a = lo;
    ctx->b = hi;
    ctx->has_filter = ctx->has_count = false;
    int32_t nf = 0;
    pfe_status st = pfe_solve(ctx, &nf);
    const pfe_stats &o = ctx->stats;
    sum.iterations += o.iterations;
    sum.matvecs += o.matvecs;
    sum.seconds_filter += o.seconds_filter;
    sum.seconds_orth += o.seconds_orth;
    sum.seconds_rr += o.seconds_rr;
    sum.fp64_sweeps += o.fp64_sweeps;
    sum.filter_launches += o.filter_launches;
    sum.filter_col_steps += o.filter_col_steps;
    sum.filter_col_steps_f32 += o.filter_col_steps_f32;
    sum.filter_col_steps_forced += o.filter_col_steps_forced;
    sum.seconds_filter_f32 += o.seconds_filter_f32;
    sum.restarts += o.restarts;
    sum.cholqr_shifts += o.cholqr_shifts;
    sum.width = std::max(sum.width, o.width);
    sum.basis = std::max(sum.basis, o.basis);
    sum.degree = std::max(sum.degree, o.degree);
    sum.count_estimate += o.count_estimate;
    sum.window_estimate += o.window_estimate;
    sum.filter_shape_f64 = o.filter_shape_f64;
    sum.filter_shape_f32 = o.filter_shape_f32;
    if (st != PFE_OK && st != PFE_E_CAPACITY) {
      ctx->a = a;
      ctx->b = b;
      ctx->has_filter = ctx->has_count = false;
      return st;  // the slice's message stays in pfe_last_error
    }
    if (st == PFE_E_CAPACITY) worst = st;
    if (nf == 0) continue;
    // grow the accumulation buffer (row-major n x ldacc) if needed
    if (used + nf > cap) {
      const int64_t ncap = std::max<int64_t>(used + nf, cap * 3 / 2 + 64);
      const int64_t nld = (ncap + 3) / 4 * 4;
      SL_RESERVE(double, nb, *tmpb, (size_t)n * nld);
      if (used > 0) {
        std::vector<int32_t> all(used);
        std::iota(all.begin(), all.end(), 0);
        SL_RESERVE(int32_t, didx, ctx->w_idx, (size_t)used);
        PFE_CUDA_TRY(ctx, cudaMemcpyAsync(didx, all.data(), sizeof(int32_t) * used, cudaMemcpyHostToDevice, s));
        launch_gather_cols(n, (int32_t)used, acc->as<double>(), ldacc, nb, nld, didx, s);
        PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
      }
      std::swap(*acc, *tmpb);
      cap = nld;
      ldacc = nld;
    }
    SL_RESERVE(int32_t, didx, ctx->w_idx, (size_t)nf);
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(didx, ctx->result_cols.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
    // columns result_cols of L -> columns used..used+nf of the accumulation buffer
    launch_gather_cols(n, nf, ctx->L.as<double>(), ctx->ldq, acc->as<double>() + used, ldacc, didx, s);
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    PFE_TRY(sl_error(ctx, "slice gather"));
    for (int32_t j = 0; j < nf; ++j) pairs.push_back(Pair{ctx->result_lam[j], ctx->result_res[j], i, used + j});
    used += nf;
  }
  ctx->a = a;
  ctx->b = b;
  ctx->has_filter = ctx->has_count = false;
  // ---- merge at every interior edge
  std::vector<char> drop(pairs.size(), 0);
  const Bsr<double> Hb = solver_bsr_H(ctx);
  for (int32_t i = 1; i < S; ++i) {
    std::vector<int32_t> zone;
    for (size_t p = 0; p < pairs.size(); ++p)
      if (!drop[p] && (pairs[p].slice == i - 1 || pairs[p].slice == i) && std::fabs(pairs[p].lam - e[i]) <= 2 * delta)
        zone.push_back((int32_t)p);
    bool both = false;
    for (int32_t p : zone)
      for (int32_t q : zone) both = both || (pairs[p].slice != pairs[q].slice);
    if (!both) continue;
    const int32_t z = (int32_t)zone.size();
    const int64_t ldz = (z + 3) / 4 * 4;
    SL_RESERVE(double, W, ctx->w_X, (size_t)n * ldz);
    SL_RESERVE(double, Q, ctx->w_Y, (size_t)n * ldz);
    SL_RESERVE(double, HQ, ctx->w_W, (size_t)n * ldz);
    SL_RESERVE(double, sm, ctx->w_small, 4 * (size_t)z * z + 4 * (size_t)z + 8);
    double *G = sm, *Sv = G + (size_t)z * z, *ev = Sv + (size_t)z * z, *r2 = ev + z;
    SL_RESERVE(double, gw, ctx->w_gram, gram_work(n, z, z, false));
    SL_RESERVE(double, red, ctx->w_red, colreduce_work(n, z));
    SL_RESERVE(int, info, ctx->w_info, 4);
    std::vector<int32_t> cols(z);
    for (int32_t t = 0; t < z; ++t) cols[t] = (int32_t)pairs[zone[t]].col;
    SL_RESERVE(int32_t, didx, ctx->w_idx, (size_t)z);
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(didx, cols.data(), sizeof(int32_t) * z, cudaMemcpyHostToDevice, s));
    launch_gather_cols(n, z, acc->as<double>(), ldacc, W, ldz, didx, s);
    // W^T W = S diag(ev) S^T; keep the directions with ev > 1/2, scaled by ev^{-1/2}
    launch_gram(n, z, z, W, ldz, W, ldz, 1.0, 0.0, G, z, false, gw, s);
    int lw = 0;
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, z, G,
                                                    z, ev, &lw));
    SL_RESERVE(double, work, ctx->w_cs_work, (size_t)std::max(lw, 1));
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, z, G, z, ev,
                                         work, lw, info));
    std::vector<double> hev(z), hS((size_t)z * z);
    int hinfo = 0;
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hev.data(), ev, sizeof(double) * z, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hS.data(), G, sizeof(double) * z * z, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hinfo != 0) return pfe_fail(ctx, PFE_E_CUDA, "cusolverDnDsyevd did not converge (slice merge)");
    std::vector<double> hB;  // z x r col-major: S_r diag(ev_r^{-1/2})
    int32_t r = 0;
    for (int32_t c = 0; c < z; ++c)
      if (hev[c] > 0.5) {
        for (int32_t t = 0; t < z; ++t) hB.push_back(hS[(size_t)c * z + t] / std::sqrt(hev[c]));
        ++r;
      }
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(Sv, hB.data(), sizeof(double) * hB.size(), cudaMemcpyHostToDevice, s));
    launch_update(n, r, z, W, ldz, Sv, z, 1.0, 0.0, Q, ldz, s);  // orthonormal basis of the joint span
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));                  // hB must outlive its copy
    // Rayleigh-Ritz with H on Q
    launch_bsr_step<double>(Hb, MODE_SPMM, r, ldz, Q, nullptr, HQ, nullptr, 1.0, 0.0, 0.0, 0.0, s);
    launch_gram(n, r, r, Q, ldz, HQ, ldz, 1.0, 0.0, G, r, false, gw, s);
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, r, G,
                                                    r, ev, &lw));
    SL_RESERVE(double, work2, ctx->w_cs_work, (size_t)std::max(lw, 1));
    PFE_SOLVER_TRY(ctx, cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, r, G, r, ev,
                                         work2, lw, info));
    launch_update(n, r, r, Q, ldz, G, r, 1.0, 0.0, W, ldz, s);  // Ritz vectors U = Q Y (into W)
    launch_bsr_step<double>(Hb, MODE_SPMM, r, ldz, W, nullptr, HQ, nullptr, 1.0, 0.0, 0.0, 0.0, s);
    launch_col_resid2(n, r, HQ, W, ldz, ev, r2, red, s);
    std::vector<double> lam(r), rr(r);
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(lam.data(), ev, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(rr.data(), r2, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hinfo != 0) return pfe_fail(ctx, PFE_E_CUDA, "cusolverDnDsyevd did not converge (slice merge)");
    PFE_TRY(sl_error(ctx, "slice merge"));
    // the merged pairs overwrite the zone's columns (r <= z)
    for (int32_t t = 0; t < z; ++t) drop[zone[t]] = 1;
    std::vector<int32_t> dst(r);
    for (int32_t t = 0; t < r; ++t) dst[t] = cols[t];
    // scatter W[:, t] -> acc[:, cols[t]]: gather with identity indices into a compact copy, column by column
    for (int32_t t = 0; t < r; ++t) {
      int32_t one = t;
      PFE_CUDA_TRY(ctx, cudaMemcpyAsync(didx, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
      launch_gather_cols(n, 1, W, ldz, acc->as<double>() + dst[t], ldacc, didx, s);
      PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // `one` must outlive its copy
      pairs.push_back(Pair{lam[t], std::sqrt(std::max(rr[t], 0.0)), -1, dst[t]});
      drop.push_back(0);
    }
    PFE_TRY(sl_error(ctx, "slice merge scatter"));
  }
  // ---- results: every kept pair inside [a, b], ascending
  std::vector<int32_t> keep;
  for (size_t p = 0; p < pairs.size(); ++p)
    if (!drop[p] && pairs[p].lam >= a && pairs[p].lam <= b) keep.push_back((int32_t)p);
  std::sort(keep.begin(), keep.end(), [&](int32_t x, int32_t y) { return pairs[x].lam < pairs[y].lam; });
  std::swap(ctx->L, *acc);
  ctx->ldq = ldacc;
  ctx->result_cols.clear();
  ctx->result_lam.clear();
  ctx->result_res.clear();
  double mr = 0.0;
  for (int32_t p : keep) {
    ctx->result_cols.push_back((int32_t)pairs[p].col);
    ctx->result_lam.push_back(pairs[p].lam);
    ctx->result_res.push_back(pairs[p].res);
    mr = std::max(mr, pairs[p].res / ctx->lmax);
  }
  ctx->n_found = (int32_t)keep.size();
  ctx->has_result = true;
  sum.n_found = ctx->n_found;
  sum.lambda_max = ctx->lmax;
  sum.max_residual = mr;
  sum.status = (int32_t)worst;
  sum.seconds_total = solver_now() - t_start;
  sum.kernel_launches = launch_count() - ctx->launch_base;
  sum.slices = S;
  ctx->stats = sum;
  if (n_found) *n_found = ctx->n_found;
  if (worst != PFE_OK) return pfe_fail(ctx, worst, "a slice's subspace could not certify completeness");
  return PFE_OK;
}
