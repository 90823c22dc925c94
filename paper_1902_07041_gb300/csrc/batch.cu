// Batched solves of independent samples (the realisations of Sec. 4.2): every sample's
// filtered subspace iteration advances in lockstep, and the filter (Alg. 2) of all samples runs
// as ONE persistent kernel per Chebyshev step.  Its warps walk a device-resident work list of
// (sample, atom, column chunk) items, so samples of uneven size share the GPU evenly.  The m_max
// step launches of one filter application are captured once into a CUDA graph and replayed each
// iteration; the per-sample descriptors (active column counts, rotating buffer pointers) live in
// device memory and are refreshed before each replay.  A CUDA-graph replay launches each step for a
// few microseconds of overhead against milliseconds of work, so the steps stay separate launches and
// no grid-wide barrier is needed between them.  An autotuner picks the column tile
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

// Chebyshev step `step` for every sample with step < m (its own degree m and coefficients):
//   step 0:  t_1 = A x / 2,            y = g_0 x + g_1 t_1
//   step j:  t_{j+1} = A t_j - t_{j-1}, and y += g_j t_j + g_{j+1} t_{j+1} when j is even, nothing when
//            j is odd unless it is the sample's last step (then y += g_m t_m): y is read and written every
//            other step, as in the single-context filter.
// Buffer rotation as in the single-context filter: step 1 reads (t_0 = X, t_1 = b0) and writes b1;
// step j >= 2 reads the pair (b0, b1) in alternating roles and overwrites t_{j-1}.
// Samples whose filter operator has the rank-1 form (u, dg set) take 6 FMAs per off-diagonal block and
// column; the others the full 3x3 blocks.  Each warp walks its items in increasing order, so its sample
// index only moves forward: a cursor replaces a search per item.
template <int CPL>
__global__ void __launch_bounds__(256) k_batch_step(const BatchDesc *__restrict__ desc, int32_t nsamp,
                                                    const int64_t *__restrict__ total_items, int32_t step) {
  const int64_t total = *total_items;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int smp = 0;
  for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < total; item += nwarps) {
    while (smp + 1 < nsamp && desc[smp + 1].item_begin <= item) ++smp;
    const BatchDesc &d = desc[smp];
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
    if (d.u) {
      // rank-1 form: diagonal block (xx, xy, xz, yy, yz, zz), then -u u^T per neighbour
      const double *g = d.dg + 6 * atom;
      const double dxx = g[0], dxy = g[1], dxz = g[2], dyy = g[3], dyz = g[4], dzz = g[5];
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc[0][c] = acc[1][c] = acc[2][c] = 0.0;
      if (on) {
        const double *xr = Xin + 3 * atom * d.ld + c0;
        double x0[CPL], x1[CPL], x2[CPL];
        ld2(xr, x0);
        ld2(xr + d.ld, x1);
        ld2(xr + 2 * d.ld, x2);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          acc[0][c] = fma(dxx, x0[c], fma(dxy, x1[c], dxz * x2[c]));
          acc[1][c] = fma(dxy, x0[c], fma(dyy, x1[c], dyz * x2[c]));
          acc[2][c] = fma(dxz, x0[c], fma(dyz, x1[c], dzz * x2[c]));
        }
      }
      const int p0 = d.rp1[atom], p1 = d.rp1[atom + 1];
      for (int p = p0; p < p1; ++p) {
        const int64_t j = d.ci1[p];
        const double u0 = d.u[3 * (int64_t)p], u1 = d.u[3 * (int64_t)p + 1], u2 = d.u[3 * (int64_t)p + 2];
        if (on) {
          const double *xr = Xin + 3 * j * d.ld + c0;
          double x0[CPL], x1[CPL], x2[CPL];
          ld2(xr, x0);
          ld2(xr + d.ld, x1);
          ld2(xr + 2 * d.ld, x2);
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const double sd = fma(u0, x0[c], fma(u1, x1[c], u2 * x2[c]));
            acc[0][c] = fma(-sd, u0, acc[0][c]);
            acc[1][c] = fma(-sd, u1, acc[1][c]);
            acc[2][c] = fma(-sd, u2, acc[2][c]);
          }
        }
      }
    } else {
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
    }
    if (!on) continue;
    const bool even = step > 0 && (step % 2) == 0;
    const bool touch_y = step == 0 || even || step == d.m - 1;
    const double ga = (step == 0) ? d.coef[0] : d.coef[step], gb = d.coef[step + 1];
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
          y[c] = fma(gb, z[c], ga * x[c]);
        }
      } else {
        double w[CPL];
        ld2(Wprev + off, w);
#pragma unroll
        for (int c = 0; c < CPL; ++c) z[c] = acc[r][c] - w[c];
        if (touch_y) {
          ld2(d.Y + off, y);
          if (even) {
            double xo[CPL];  // this step's input rows of this atom: g_j t_j joins y one step late
            ld2(Xin + off, xo);
#pragma unroll
            for (int c = 0; c < CPL; ++c) y[c] = fma(ga, xo[c], fma(gb, z[c], y[c]));
          } else {
#pragma unroll
            for (int c = 0; c < CPL; ++c) y[c] = fma(gb, z[c], y[c]);
          }
        }
      }
      st2(Z + off, z);
      if (touch_y) st2(d.Y + off, y);
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
