// Batched solves of independent samples (the realisations of Sec. 4.2): every sample's
// filtered subspace iteration advances in lockstep, and the filter (Alg. 2) of all samples runs
// as ONE persistent kernel per Chebyshev step.  Its warps walk a device-resident work list of
// (sample, atom, column chunk) items, so samples of uneven size share the GPU evenly.  The m_max
// step launches of one filter application are captured once into a CUDA graph and replayed each
// iteration; the per-sample descriptors (active column counts, rotating buffer pointers) live in
// device memory and are refreshed before each replay.  An autotuner picks the column tile
// (32 or 64 columns per warp) and the persistent grid size by timing the candidates.
#include <cmath>

#include "pfe_internal.h"

namespace pfe {

namespace {

__device__ __forceinline__ void ld2(const double *p, double (&v)[2]) {
  const double2 t = *reinterpret_cast<const double2 *>(p);
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void ld2(const double *p, double (&v)[1]) { v[0] = *p; }
__device__ __forceinline__ void st2(double *p, const double (&v)[2]) {
  *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void st2(double *p, const double (&v)[1]) { *p = v[0]; }

// Chebyshev step `step` (0 = t_1 and y = g0 x + g1 t_1; j >= 1: t_{j+1} = A t_j - t_{j-1},
// y += g_{j+1} t_{j+1}) for every sample with step < m.  Buffer rotation as in the single-context
// filter: step 1 reads (t_0 = X, t_1 = b0) and writes b1; step j >= 2 reads the pair
// (b0, b1) in alternating roles and overwrites t_{j-1}.
template <int CPL>
__global__ void __launch_bounds__(256) k_batch_step(const BatchDesc *__restrict__ desc, int32_t nsamp,
                                                    const int64_t *__restrict__ total_items, int32_t step) {
  const int64_t total = *total_items;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < total; item += nwarps) {
    // sample of this item: last s with item_begin <= item (binary search over the prefix)
    int lo = 0, hi = nsamp - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (desc[mid].item_begin <= item) lo = mid;
      else hi = mid - 1;
    }
    const BatchDesc &d = desc[lo];
    if (step >= d.m) continue;
    const int64_t local = item - d.item_begin;
    const int64_t atom = local / d.nchunk;
    const int chunk = (int)(local - atom * d.nchunk);
    const int c0 = (chunk * 32 + lane) * CPL;
    const bool on = c0 < d.k;
    const double *Xin;
    const double *Wprev;
    double *Z;
    if (step == 0) {
      Xin = d.X; Wprev = nullptr; Z = d.b0;
    } else if (step == 1) {
      Xin = d.b0; Wprev = d.X; Z = d.b1;
    } else {
      Xin = (step % 2 == 0) ? d.b1 : d.b0;
      Z = (step % 2 == 0) ? d.b0 : d.b1;
      Wprev = Z;
    }
    double acc[3][CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) acc[0][c] = acc[1][c] = acc[2][c] = 0.0;
    const int p0 = d.rp[atom], p1 = d.rp[atom + 1];
    for (int p = p0; p < p1; ++p) {
      const int64_t j = d.ci[p];
      double a[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) a[t] = d.vals[9 * (int64_t)p + t];
      if (on) {
        const double *xr = Xin + 3 * j * d.ld + c0;
        double x0[CPL], x1[CPL], x2[CPL];
        ld2(xr, x0);
        ld2(xr + d.ld, x1);
        ld2(xr + 2 * d.ld, x2);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          acc[0][c] = fma(a[0], x0[c], fma(a[1], x1[c], fma(a[2], x2[c], acc[0][c])));
          acc[1][c] = fma(a[3], x0[c], fma(a[4], x1[c], fma(a[5], x2[c], acc[1][c])));
          acc[2][c] = fma(a[6], x0[c], fma(a[7], x1[c], fma(a[8], x2[c], acc[2][c])));
        }
      }
    }
    if (!on) continue;
    const double g0 = d.coef[0], g1 = d.coef[step + 1];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int64_t off = (3 * atom + r) * d.ld + c0;
      double z[CPL], y[CPL];
      if (step == 0) {
        double x[CPL];
        ld2(d.X + off, x);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          z[c] = 0.5 * acc[r][c];
          y[c] = fma(g1, z[c], g0 * x[c]);
        }
      } else {
        double w[CPL];
        ld2(Wprev + off, w);
        ld2(d.Y + off, y);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          z[c] = acc[r][c] - w[c];
          y[c] = fma(g1, z[c], y[c]);
        }
      }
      st2(Z + off, z);
      st2(d.Y + off, y);
    }
  }
}

}  // namespace

void launch_batch_step(int cpl, int blocks, const BatchDesc *desc, int32_t nsamp, const int64_t *total, int32_t step,
                       cudaStream_t s) {
  if (cpl == 2)
    PFE_LAUNCH k_batch_step<2><<<blocks, 256, 0, s>>>(desc, nsamp, total, step);
  else
    PFE_LAUNCH k_batch_step<1><<<blocks, 256, 0, s>>>(desc, nsamp, total, step);
}

}  // namespace pfe
