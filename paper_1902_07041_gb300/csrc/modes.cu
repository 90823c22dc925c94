// Analysis of the computed modes (Sec. 4.4): the participation ratio of eq. (PR_def) and the
// plane-wave content of each eigenvector.  A mode q is read as N 3-vectors q_i (the three dof
// rows of atom i).
//
//   participation ratio, normalised by N:  PR = (sum_i |q_i|^2)^2 / (N sum_i |q_i|^4)
//     (1 for a mode spread evenly over the atoms, 1/N for a single atom, 2/3 for a plane wave);
//   plane-wave content for a wave vector k:  A_d = sum_i q_{i,d} e^{i k . r_i},
//     longitudinal (2/N) |k^ . A|^2 / |q|^2 and transverse (2/N) (|A|^2 - |k^ . A|^2) / |q|^2
//     (the weight of q on the plane waves sqrt(2/N) zeta sin(k . r_i) and sqrt(2/N) zeta cos(k . r_i),
//     zeta along or across k; 1 for a pure plane wave of an allowed k).
// The sums over atoms of A are a dense contraction Q_d^T E with E[i] = (cos k_w.r_i, sin k_w.r_i):
// they run on the DMMA Gram kernel.
#include <cmath>

#include "pfe_internal.h"

using namespace pfe;

namespace {

#define MODES_RESERVE(T, ptr, buf, count)                                                   \
  T *ptr = nullptr;                                                                         \
  {                                                                                         \
    cudaError_t e__ = dbuf_reserve((buf), (size_t)(count) * sizeof(T));                     \
    if (e__ != cudaSuccess)                                                                 \
      return pfe_fail(ctx, PFE_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e__)); \
    ptr = (buf).as<T>();                                                                    \
  }

constexpr int kRowsPerBlock = 8;

// partial[by][0][c] = sum |q_i|^2, partial[by][1][c] = sum |q_i|^4 over the atoms of row block by
// (grid-stride over blocks of 8 atoms); Q row-major n x ld, column c of k.
__global__ void k_mode_norms(int32_t n_atoms, int32_t k, const double *__restrict__ Q, int64_t ld, double *partial) {
  __shared__ double s2[kRowsPerBlock][32], s4[kRowsPerBlock][32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int32_t c = blockIdx.x * 32 + tx;
  double a2 = 0.0, a4 = 0.0;
  if (c < k) {
    for (int64_t i = (int64_t)blockIdx.y * kRowsPerBlock + ty; i < n_atoms; i += (int64_t)gridDim.y * kRowsPerBlock) {
      const double x = Q[(3 * i) * ld + c], y = Q[(3 * i + 1) * ld + c], z = Q[(3 * i + 2) * ld + c];
      const double w = x * x + y * y + z * z;
      a2 += w;
      a4 += w * w;
    }
  }
  s2[ty][tx] = a2;
  s4[ty][tx] = a4;
  __syncthreads();
  if (ty == 0 && c < k) {
    double t2 = 0.0, t4 = 0.0;
    for (int r = 0; r < kRowsPerBlock; ++r) {
      t2 += s2[r][tx];
      t4 += s4[r][tx];
    }
    partial[((int64_t)blockIdx.y * 2) * k + c] = t2;
    partial[((int64_t)blockIdx.y * 2 + 1) * k + c] = t4;
  }
}

// norm2[c], pr[c] from the partial sums in fixed order
__global__ void k_mode_norms_reduce(int32_t n_atoms, int32_t k, int32_t parts, const double *partial, double *norm2,
                                    double *pr) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double t2 = 0.0, t4 = 0.0;
  for (int32_t b = 0; b < parts; ++b) {
    t2 += partial[((int64_t)b * 2) * k + c];
    t4 += partial[((int64_t)b * 2 + 1) * k + c];
  }
  norm2[c] = t2;
  pr[c] = (t4 > 0.0) ? t2 * t2 / ((double)n_atoms * t4) : 0.0;
}

// E[i * lde + 2w] = cos(k_w . r_i), E[i * lde + 2w + 1] = sin(k_w . r_i)
__global__ void k_phase_matrix(int32_t n_atoms, int32_t nk, const double *__restrict__ pos,
                               const double *__restrict__ kvec, double *E, int64_t lde) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_atoms * nk) return;
  const int64_t i = t / nk;
  const int w = (int)(t - i * nk);
  const double ph = kvec[3 * w] * pos[3 * i] + kvec[3 * w + 1] * pos[3 * i + 1] + kvec[3 * w + 2] * pos[3 * i + 2];
  double sn, cs;
  sincos(ph, &sn, &cs);
  E[i * lde + 2 * w] = cs;
  E[i * lde + 2 * w + 1] = sn;
}

// The found eigenvectors, gathered in result order into a row-major n x ldt buffer, and their
// squared norms and participation ratios (device arrays of nf).
pfe_status gather_modes(pfe_ctx *ctx, double **Q, int64_t *ldt_out, double **norm2, double **pr) {
  const int64_t n = ctx->n;
  const int32_t nf = ctx->n_found;
  cudaStream_t s = ctx->stream;
  const int64_t ldt = (nf + 3) / 4 * 4;
  MODES_RESERVE(double, tmp, ctx->w_Y, (size_t)n * ldt);
  MODES_RESERVE(int32_t, idx, ctx->w_idx, (size_t)nf);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(idx, ctx->result_cols.data(), sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
  launch_gather_cols(n, nf, ctx->L.as<double>(), ctx->ldq, tmp, ldt, idx, s);
  const int32_t parts = (int32_t)std::min<int64_t>(1024, (ctx->N + kRowsPerBlock - 1) / kRowsPerBlock);
  MODES_RESERVE(double, work, ctx->w_red, (size_t)2 * parts * nf + 2 * (size_t)nf);
  double *nrm = work + (size_t)2 * parts * nf, *p = nrm + nf;
  dim3 grid((nf + 31) / 32, parts), block(32, kRowsPerBlock);
  PFE_LAUNCH k_mode_norms<<<grid, block, 0, s>>>(ctx->N, nf, tmp, ldt, work);
  PFE_LAUNCH k_mode_norms_reduce<<<(nf + 127) / 128, 128, 0, s>>>(ctx->N, nf, parts, work, nrm, p);
  *Q = tmp;
  *ldt_out = ldt;
  *norm2 = nrm;
  *pr = p;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, std::string("mode norms: ") + cudaGetErrorString(e));
  return PFE_OK;
}

}  // namespace

extern "C" {

pfe_status pfe_participation_ratio(pfe_ctx *ctx, int32_t cap, double *pr) {
  if (!ctx) return PFE_E_ARG;
  if (!pr) return pfe_fail(ctx, PFE_E_ARG, "participation_ratio: null output");
  if (!ctx->has_result) return pfe_fail(ctx, PFE_E_STATE, "no solve results");
  const int32_t nf = ctx->n_found;
  if (cap < nf) return pfe_fail(ctx, PFE_E_CAPACITY, "output capacity below the number of eigenpairs found");
  if (nf == 0) return PFE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  double *Q = nullptr, *nrm = nullptr, *dpr = nullptr;
  int64_t ldt = 0;
  PFE_TRY(gather_modes(ctx, &Q, &ldt, &nrm, &dpr));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(pr, dpr, sizeof(double) * nf, cudaMemcpyDeviceToHost, ctx->stream));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return PFE_OK;
}

pfe_status pfe_plane_wave_content(pfe_ctx *ctx, const double *pos, int32_t nk, const double *kvec, int32_t cap,
                                  double *out) {
  if (!ctx) return PFE_E_ARG;
  if (nk < 0 || (nk > 0 && (!pos || !kvec || !out))) return pfe_fail(ctx, PFE_E_ARG, "plane_wave_content: bad arguments");
  if (!ctx->has_result) return pfe_fail(ctx, PFE_E_STATE, "no solve results");
  const int32_t nf = ctx->n_found;
  if (cap < nf) return pfe_fail(ctx, PFE_E_CAPACITY, "output capacity below the number of eigenpairs found");
  std::vector<double> khat(3 * (size_t)nk);
  for (int32_t w = 0; w < nk; ++w) {
    const double kx = kvec[3 * w], ky = kvec[3 * w + 1], kz = kvec[3 * w + 2];
    const double kn = std::sqrt(kx * kx + ky * ky + kz * kz);
    if (!(kn > 0.0) || !std::isfinite(kn)) return pfe_fail(ctx, PFE_E_ARG, "plane_wave_content: zero or non-finite wave vector");
    khat[3 * w] = kx / kn;
    khat[3 * w + 1] = ky / kn;
    khat[3 * w + 2] = kz / kn;
  }
  for (int64_t i = 0; i < 3 * (int64_t)ctx->N; ++i)
    if (!std::isfinite(pos[i])) return pfe_fail(ctx, PFE_E_ARG, "plane_wave_content: non-finite position");
  if (nf == 0 || nk == 0) return PFE_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  cudaStream_t s = ctx->stream;
  double *Q = nullptr, *nrm = nullptr, *dpr = nullptr;
  int64_t ldt = 0;
  PFE_TRY(gather_modes(ctx, &Q, &ldt, &nrm, &dpr));
  const int64_t N = ctx->N, lde = (2 * (int64_t)nk + 3) / 4 * 4;
  // device: positions, wave vectors, E (N x lde), C_d (nf x 2nk col-major, d = 0..2), Gram work
  const size_t cbytes = (size_t)nf * 2 * nk;
  MODES_RESERVE(double, dev, ctx->w_W, 3 * (size_t)N + 3 * (size_t)nk + (size_t)N * lde + 3 * cbytes);
  double *dpos = dev, *dk = dpos + 3 * N, *E = dk + 3 * (size_t)nk, *C = E + (size_t)N * lde;
  MODES_RESERVE(double, gw, ctx->w_gram, gram_work(N, nf, 2 * nk, false));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(dpos, pos, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(dk, kvec, sizeof(double) * 3 * nk, cudaMemcpyHostToDevice, s));
  const int64_t tot = N * nk;
  PFE_LAUNCH k_phase_matrix<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((int32_t)N, nk, dpos, dk, E, lde);
  for (int d = 0; d < 3; ++d)  // C_d[s, 2w (+1)] = sum_i q_{i,d} (cos, sin)(k_w . r_i)
    launch_gram(N, nf, 2 * nk, Q + d * ldt, 3 * ldt, E, lde, 1.0, 0.0, C + (size_t)d * cbytes, nf, false, gw, s);
  std::vector<double> hC(3 * cbytes), hn(nf);
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hC.data(), C, sizeof(double) * 3 * cbytes, cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaMemcpyAsync(hn.data(), nrm, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
  PFE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, std::string("plane_wave_content: ") + cudaGetErrorString(e));
  for (int32_t m = 0; m < nf; ++m)
    for (int32_t w = 0; w < nk; ++w) {
      double re[3], im[3], tot2 = 0.0, lre = 0.0, lim = 0.0;
      for (int d = 0; d < 3; ++d) {
        re[d] = hC[(size_t)d * cbytes + (size_t)(2 * w) * nf + m];
        im[d] = hC[(size_t)d * cbytes + (size_t)(2 * w + 1) * nf + m];
        tot2 += re[d] * re[d] + im[d] * im[d];
        lre += khat[3 * w + d] * re[d];
        lim += khat[3 * w + d] * im[d];
      }
      const double l2 = lre * lre + lim * lim;
      const double scale = (hn[m] > 0.0) ? 2.0 / ((double)N * hn[m]) : 0.0;
      out[((size_t)m * nk + w) * 2] = scale * l2;
      out[((size_t)m * nk + w) * 2 + 1] = scale * std::max(tot2 - l2, 0.0);
    }
  return PFE_OK;
}

}  // extern "C"
