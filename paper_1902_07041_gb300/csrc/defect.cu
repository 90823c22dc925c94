// Mixed-precision filter by defect correction.
//
// For a block X with Ritz values theta (diagonal Theta) and W = H X, write Ht = (H - cI)/d,
// Theta_t = (Theta - cI)/d and Rt = Ht X - X Theta_t = (W - X Theta)/d.  With tau_j = T_j(Theta_t)
// (per column) and D_j = T_j(Ht) X - X tau_j, the three-term recurrence of Alg. 2 gives
//     D_0 = 0,  D_1 = Rt,  D_{j+1} = 2 Ht D_j - D_{j-1} + 2 Rt tau_j,
// and the filter is, exactly,
//     p(Ht) X = sum_j g_j T_j(Ht) X = X p(Theta_t) + sum_j g_j D_j.
// The first term is formed in FP64; the sum of the D_j, whose size follows the residual, runs in FP32.
// Its rounding error is then relative to ||Rt|| instead of ||X||, so a Ritz pair keeps converging
// below the FP32 noise level of the plain filter without an FP64 sweep.  (The recurrence is the one
// of Alg. 2; only the split of p(Ht) X into an FP64 and an FP32 part is new.)
//
// In one launch per step, the columns of a block may be of either kind: "defect" columns run the
// recurrence above (forcing 2 tau_j Rt), "plain" columns the plain FP32 recurrence (forcing factor
// 0 and Rt = 0), so both groups share the neighbour gathers of every step.
#include "pfe_internal.h"
#include "vec_io.cuh"

namespace pfe {
namespace {

// One step of the recurrence with forcing, FP32, warp per (atom, column chunk) as the rank-1 step
// kernel (MINB resident CTAs per SM: 5, or 6 when the tuner chose shape 11 for the plain step):
//   Z = A X - W + fs[c] F                       (X = D_j, W = D_{j-1}, may alias Z; F = Rt)
//   MODE_STEP:     Y += g1 Z  when Y is given   (odd steps: only the last one)
//   MODE_STEP_ACC: Y += g0 X + g1 Z             (even steps: the input's term one step late)
// R1: the operator's rank-1 form (u, dg); otherwise its full 3x3 blocks (vals).
template <int CPL, int MODE, bool R1, int MINB>
__global__ void __launch_bounds__(256, MINB) k_defect_step(int32_t n_atoms, const int32_t *__restrict__ rp,
                                                        const int32_t *__restrict__ ci, const float *__restrict__ vals,
                                                        const float *__restrict__ u, const float *__restrict__ dg,
                                                        int32_t k, int64_t ld, int32_t nchunk,
                                                        const float *__restrict__ X, const float *W, float *Z,
                                                        float *Y, const float *__restrict__ F,
                                                        const float *__restrict__ fs, float g0, float g1) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t atom = gw / nchunk;
  if (atom >= n_atoms) return;
  const int chunk = (int)(gw - atom * nchunk);
  const int c0 = (chunk * 32 + lane) * CPL;
  const bool on = c0 < k;
  float acc[3][CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) acc[0][c] = acc[1][c] = acc[2][c] = 0.f;
  if (R1) {
    const float *d = dg + 6 * atom;
    const float dxx = __ldg(d), dxy = __ldg(d + 1), dxz = __ldg(d + 2), dyy = __ldg(d + 3), dyz = __ldg(d + 4),
                dzz = __ldg(d + 5);
    if (on) {
      const float *xr = X + 3 * atom * ld + c0;
      float x0[CPL], x1[CPL], x2[CPL];
      ldg_n(xr, x0);
      ldg_n(xr + ld, x1);
      ldg_n(xr + 2 * ld, x2);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        acc[0][c] = fmaf(dxx, x0[c], fmaf(dxy, x1[c], dxz * x2[c]));
        acc[1][c] = fmaf(dxy, x0[c], fmaf(dyy, x1[c], dyz * x2[c]));
        acc[2][c] = fmaf(dxz, x0[c], fmaf(dyz, x1[c], dzz * x2[c]));
      }
    }
    const int p0 = __ldg(rp + atom), p1 = __ldg(rp + atom + 1);
    for (int p = p0; p < p1; ++p) {
      const int64_t j = __ldg(ci + p);
      const float u0 = __ldg(u + 3 * (int64_t)p), u1 = __ldg(u + 3 * (int64_t)p + 1), u2 = __ldg(u + 3 * (int64_t)p + 2);
      if (on) {
        const float *xr = X + 3 * j * ld + c0;
        float x0[CPL], x1[CPL], x2[CPL];
        ldg_n(xr, x0);
        ldg_n(xr + ld, x1);
        ldg_n(xr + 2 * ld, x2);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const float sd = fmaf(u0, x0[c], fmaf(u1, x1[c], u2 * x2[c]));
          acc[0][c] = fmaf(-sd, u0, acc[0][c]);
          acc[1][c] = fmaf(-sd, u1, acc[1][c]);
          acc[2][c] = fmaf(-sd, u2, acc[2][c]);
        }
      }
    }
  } else {
    const int p0 = __ldg(rp + atom), p1 = __ldg(rp + atom + 1);
    for (int p = p0; p < p1; ++p) {
      const int64_t j = __ldg(ci + p);
      const float *v = vals + 9 * (int64_t)p;
      float a[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) a[t] = __ldg(v + t);
      if (on) {
        const float *xr = X + 3 * j * ld + c0;
        float x0[CPL], x1[CPL], x2[CPL];
        ldg_n(xr, x0);
        ldg_n(xr + ld, x1);
        ldg_n(xr + 2 * ld, x2);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          acc[0][c] = fmaf(a[0], x0[c], fmaf(a[1], x1[c], fmaf(a[2], x2[c], acc[0][c])));
          acc[1][c] = fmaf(a[3], x0[c], fmaf(a[4], x1[c], fmaf(a[5], x2[c], acc[1][c])));
          acc[2][c] = fmaf(a[6], x0[c], fmaf(a[7], x1[c], fmaf(a[8], x2[c], acc[2][c])));
        }
      }
    }
  }
  if (!on) return;
  float s[CPL];
  ldg_n(fs + c0, s);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int64_t off = (3 * atom + r) * ld + c0;
    float z[CPL], w[CPL], f[CPL];
    ld_n(W + off, w);
    ldg_n(F + off, f);
#pragma unroll
    for (int c = 0; c < CPL; ++c) z[c] = fmaf(s[c], f[c], acc[r][c] - w[c]);
    st_n(Z + off, z);
    if (MODE == MODE_STEP && Y != nullptr) {
      float y[CPL];
      ld_n(Y + off, y);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fmaf(g1, z[c], y[c]);
      st_n(Y + off, y);
    } else if (MODE == MODE_STEP_ACC) {
      float y[CPL], x[CPL];
      ld_n(Y + off, y);
      ldg_n(X + off, x);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fmaf(g0, x[c], fmaf(g1, z[c], y[c]));
      st_n(Y + off, y);
    }
  }
}

// Start of a mixed block (row-major, act columns, the first k_d of them defect columns):
//   defect columns: Rt = (W - theta X) / d;  X32 = 0 (D_0);  B = Rt (D_1);  F = Rt;  Y32 = g1 Rt
//   plain columns:  X32 = X (t_0, rounded);  F = 0
// One thread per (row, column).
__global__ void k_defect_prep(int64_t n, int32_t act, int32_t kd, const double *__restrict__ X,
                              const double *__restrict__ W, int64_t ld, const double *__restrict__ theta,
                              double inv_d, double g1, float *X32, float *B, float *F, float *Y32) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * act) return;
  const int64_t i = idx / act;
  const int32_t c = (int32_t)(idx - i * act);
  const int64_t off = i * ld + c;
  if (c < kd) {
    const double r = (W[off] - theta[c] * X[off]) * inv_d;
    const float rf = (float)r;
    X32[off] = 0.f;
    B[off] = rf;
    F[off] = rf;
    Y32[off] = (float)(g1 * r);
  } else {
    X32[off] = (float)X[off];
    F[off] = 0.f;
  }
}

// End of a mixed block: Y = pth[c] X + Y32 (pth = p(theta_t) for defect columns, 0 for plain ones).
__global__ void k_defect_combine(int64_t n, int32_t act, const double *__restrict__ X, int64_t ld,
                                 const double *__restrict__ pth, const float *__restrict__ Y32, double *Y) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * act) return;
  const int64_t i = idx / act;
  const int32_t c = (int32_t)(idx - i * act);
  const int64_t off = i * ld + c;
  Y[off] = fma(pth[c], X[off], (double)Y32[off]);
}

template <int CPL, int MINB>
void dispatch_defect_cpl(const Bsr<float> &A, int mode, int32_t k, int64_t ld, const float *X, const float *W, float *Z,
                         float *Y, const float *F, const float *fs, float g0, float g1, cudaStream_t s) {
  const int32_t nchunk = (k + 32 * CPL - 1) / (32 * CPL);
  const int64_t blocks = ((int64_t)A.n_atoms * nchunk * 32 + 255) / 256;
  const bool r1 = A.u != nullptr;
  const int32_t *rp = r1 ? A.rp1 : A.rp;
  const int32_t *ci = r1 ? A.ci1 : A.ci;
#define PFE_DEFECT_LAUNCH(M, R)                                                                           \
  PFE_LAUNCH k_defect_step<CPL, M, R, MINB><<<(unsigned)blocks, 256, 0, s>>>(A.n_atoms, rp, ci, A.vals, A.u, A.dg, k, ld, \
                                                                       nchunk, X, W, Z, Y, F, fs, g0, g1)
  if (mode == MODE_STEP_ACC) {
    if (r1) PFE_DEFECT_LAUNCH(MODE_STEP_ACC, true);
    else PFE_DEFECT_LAUNCH(MODE_STEP_ACC, false);
  } else {
    if (r1) PFE_DEFECT_LAUNCH(MODE_STEP, true);
    else PFE_DEFECT_LAUNCH(MODE_STEP, false);
  }
#undef PFE_DEFECT_LAUNCH
}

bool al16(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) % 16) == 0; }

}  // namespace

void launch_defect_step(const Bsr<float> &A, int mode, int32_t k, int64_t ld, const float *X, const float *W, float *Z,
                        float *Y, const float *F, const float *fs, float g0, float g1, cudaStream_t s, bool six_ctas) {
  if (k <= 0 || A.n_atoms <= 0) return;
  const bool v4 = ld % 4 == 0 && al16(X) && al16(W) && al16(Z) && al16(Y) && al16(F) && al16(fs) && k > 64;
  if (v4 && six_ctas)
    dispatch_defect_cpl<4, 6>(A, mode, k, ld, X, W, Z, Y, F, fs, g0, g1, s);
  else if (v4)
    dispatch_defect_cpl<4, 5>(A, mode, k, ld, X, W, Z, Y, F, fs, g0, g1, s);
  else
    dispatch_defect_cpl<1, 5>(A, mode, k, ld, X, W, Z, Y, F, fs, g0, g1, s);
}

void launch_defect_prep(int64_t n, int32_t act, int32_t kd, const double *X, const double *W, int64_t ld,
                        const double *theta, double inv_d, double g1, float *X32, float *B, float *F, float *Y32,
                        cudaStream_t s) {
  const int64_t tot = n * act;
  if (tot <= 0) return;
  PFE_LAUNCH k_defect_prep<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, act, kd, X, W, ld, theta, inv_d, g1, X32, B,
                                                                         F, Y32);
}

void launch_defect_combine(int64_t n, int32_t act, const double *X, int64_t ld, const double *pth, const float *Y32,
                           double *Y, cudaStream_t s) {
  const int64_t tot = n * act;
  if (tot <= 0) return;
  PFE_LAUNCH k_defect_combine<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, act, X, ld, pth, Y32, Y);
}

}  // namespace pfe
