// The fused Chebyshev step on the rank-1 form of a central-force Hessian.
//
// For a spring network every off-diagonal block of H is H_ij = -k_ij r r^T / sqrt(m_i m_j)
// (eqs. (1)-(2)): a negative semidefinite rank-1 matrix.  The filter operator
// A = (2/d)(H - cI) then has off-diagonal blocks A_ij = -u u^T with u = sqrt(2 k_ij / (d sqrt(m_i m_j))) r,
// and the product with a neighbour's three rows costs s = u . x_j (3 FMAs) and acc -= s u
// (3 FMAs) per column instead of the 9 FMAs of a full 3x3 block; it reads 3 values instead of 9.
// The diagonal blocks stay full (symmetric, 6 values).  The block compression is the one the
// paper's outlook proposes for the Hessian's 3x3 structure (Sec. 5).
//
// Layout: rp1/ci1 is the BSR pattern without the diagonal blocks, u holds 3 values per
// off-diagonal block, dg 6 per atom (xx, xy, xz, yy, yz, zz).  The mapping of warps, lanes and
// columns is the one of the BSR step kernel (warp per (atom, column chunk), CPL columns a lane).
#include "pfe_internal.h"
#include "vec_io.cuh"

namespace pfe {
namespace {

template <typename T, int CPL, int MODE, int UNROLL, int MINB>
__global__ void __launch_bounds__(256, MINB) k_r1_step(int32_t n_atoms, const int32_t *__restrict__ rp1,
                                                       const int32_t *__restrict__ ci1, const T *__restrict__ u,
                                                       const T *__restrict__ dg, int32_t k, int64_t ld, int32_t nchunk,
                                                       const T *__restrict__ X, const T *W, T *Z, T *Y, T alpha,
                                                       T beta, T g0, T g1) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t atom = gw / nchunk;
  if (atom >= n_atoms) return;
  const int chunk = (int)(gw - atom * nchunk);
  const int c0 = (chunk * 32 + lane) * CPL;
  const bool on = c0 < k;
  T xo[3][CPL], acc[3][CPL];
  {
    const T *d = dg + 6 * atom;
    const T dxx = __ldg(d), dxy = __ldg(d + 1), dxz = __ldg(d + 2), dyy = __ldg(d + 3), dyz = __ldg(d + 4),
            dzz = __ldg(d + 5);
    if (on) {
      const T *xr = X + 3 * atom * ld + c0;
      ldg_n(xr, xo[0]);
      ldg_n(xr + ld, xo[1]);
      ldg_n(xr + 2 * ld, xo[2]);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        acc[0][c] = fma(dxx, xo[0][c], fma(dxy, xo[1][c], dxz * xo[2][c]));
        acc[1][c] = fma(dxy, xo[0][c], fma(dyy, xo[1][c], dyz * xo[2][c]));
        acc[2][c] = fma(dxz, xo[0][c], fma(dyz, xo[1][c], dzz * xo[2][c]));
      }
    }
  }
  const int p0 = __ldg(rp1 + atom), p1 = __ldg(rp1 + atom + 1);
  for (int p = p0; p < p1; p += UNROLL) {
    T uu[UNROLL][3];
    T x[UNROLL][3][CPL];
    bool has[UNROLL];
#pragma unroll
    for (int v = 0; v < UNROLL; ++v) {
      has[v] = (p + v) < p1;
      const int pv = has[v] ? p + v : p;
      const int64_t j = __ldg(ci1 + pv);
      uu[v][0] = __ldg(u + 3 * (int64_t)pv);
      uu[v][1] = __ldg(u + 3 * (int64_t)pv + 1);
      uu[v][2] = __ldg(u + 3 * (int64_t)pv + 2);
      if (on) {
        const T *xr = X + 3 * j * ld + c0;
        ldg_n(xr, x[v][0]);
        ldg_n(xr + ld, x[v][1]);
        ldg_n(xr + 2 * ld, x[v][2]);
      }
    }
    if (on) {
#pragma unroll
      for (int v = 0; v < UNROLL; ++v) {
        if (!has[v]) continue;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const T sdot = fma(uu[v][0], x[v][0][c], fma(uu[v][1], x[v][1][c], uu[v][2] * x[v][2][c]));
          acc[0][c] = fma(-sdot, uu[v][0], acc[0][c]);
          acc[1][c] = fma(-sdot, uu[v][1], acc[1][c]);
          acc[2][c] = fma(-sdot, uu[v][2], acc[2][c]);
        }
      }
    }
  }
  if (!on) return;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int64_t off = (3 * atom + r) * ld + c0;
    T z[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) z[c] = alpha * acc[r][c];
    if (MODE == MODE_STEP || MODE == MODE_STEP_ACC || MODE == MODE_ADJ) {
      T w[CPL];
      ld_n(W + off, w);
#pragma unroll
      for (int c = 0; c < CPL; ++c) z[c] = fma(beta, w[c], z[c]);
    }
    if (MODE == MODE_ADJ) {
      T y[CPL];
      ld_n(Y + off, y);
#pragma unroll
      for (int c = 0; c < CPL; ++c) z[c] = fma(g0, y[c], z[c]);
    }
    st_n(Z + off, z);
    if (MODE == MODE_FIRST) {
      T y[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g1, z[c], g0 * xo[r][c]);
      st_n(Y + off, y);
    } else if (MODE == MODE_STEP && Y != nullptr) {
      T y[CPL];
      ld_n(Y + off, y);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g1, z[c], y[c]);
      st_n(Y + off, y);
    } else if (MODE == MODE_STEP_ACC) {
      // also the pending term g0 t_j: this atom's rows of X again (cache hits), so that they need
      // not stay in registers through the neighbour loop
      T y[CPL], x[CPL];
      ld_n(Y + off, y);
      ldg_n(X + off, x);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g0, x[c], fma(g1, z[c], y[c]));
      st_n(Y + off, y);
    }
  }
}

template <typename T, int CPL, int UNROLL, int MINB>
void dispatch_r1_mode(const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z, T *Y, T alpha,
                      T beta, T g0, T g1, cudaStream_t s) {
  const int32_t nchunk = (k + 32 * CPL - 1) / (32 * CPL);
  const int64_t blocks = ((int64_t)A.n_atoms * nchunk * 32 + 255) / 256;
#define PFE_R1_LAUNCH(M)                                                                                    \
  PFE_LAUNCH k_r1_step<T, CPL, M, UNROLL, MINB><<<(unsigned)blocks, 256, 0, s>>>(                           \
      A.n_atoms, A.rp1, A.ci1, A.u, A.dg, k, ld, nchunk, X, W, Z, Y, alpha, beta, g0, g1)
  if (mode == MODE_SPMM)
    PFE_R1_LAUNCH(MODE_SPMM);
  else if (mode == MODE_FIRST)
    PFE_R1_LAUNCH(MODE_FIRST);
  else if (mode == MODE_ADJ)
    PFE_R1_LAUNCH(MODE_ADJ);
  else if (mode == MODE_STEP_ACC)
    PFE_R1_LAUNCH(MODE_STEP_ACC);
  else
    PFE_R1_LAUNCH(MODE_STEP);
#undef PFE_R1_LAUNCH
}

template <typename T, int CPL>
void dispatch_r1_variant(int variant, const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z,
                         T *Y, T alpha, T beta, T g0, T g1, cudaStream_t s) {
  switch (variant) {
    case 1: dispatch_r1_mode<T, CPL, 1, 5>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
    case 2: dispatch_r1_mode<T, CPL, 2, 1>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
    case 4: dispatch_r1_mode<T, CPL, 1, 6>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
    default: dispatch_r1_mode<T, CPL, 1, 1>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
  }
}

// Rank-1 form of A = alpha (H - shift I).  One thread per atom row; every row holds exactly one
// diagonal block.  An off-diagonal block that is not -u u^T to 1e-12 of its largest entry sets *bad.
__global__ void k_build_r1(int32_t n_atoms, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ H, double alpha, double shift, int32_t *rp1, int32_t *ci1,
                           double *u64, double *dg64, float *u32, float *dg32, int32_t *bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_atoms) return;
  const int32_t p0 = rp[i], p1 = rp[i + 1];
  int64_t q = (int64_t)p0 - i;
  rp1[i] = (int32_t)q;
  if (i == n_atoms - 1) rp1[n_atoms] = p1 - n_atoms;
  for (int32_t p = p0; p < p1; ++p) {
    const double *h = H + 9 * (int64_t)p;
    if (ci[p] == i) {
      const double d[6] = {alpha * (h[0] - shift), alpha * h[1], alpha * h[2], alpha * (h[4] - shift), alpha * h[5],
                           alpha * (h[8] - shift)};
      for (int t = 0; t < 6; ++t) {
        dg64[6 * i + t] = d[t];
        if (dg32) dg32[6 * i + t] = (float)d[t];
      }
      continue;
    }
    // -h = kappa r r^T: u_r = sqrt(alpha) (-h)[r][a] / sqrt((-h)[a][a]), a the largest diagonal entry
    int a = 0;
    if (-h[4] > -h[3 * a + a]) a = 1;
    if (-h[8] > -h[3 * a + a]) a = 2;
    const double haa = -h[3 * a + a];
    double hmax = 0.0;
    for (int t = 0; t < 9; ++t) hmax = fmax(hmax, fabs(h[t]));
    double uv[3] = {0.0, 0.0, 0.0};
    if (haa > 0.0) {
      const double sc = sqrt(alpha / haa);
      for (int r = 0; r < 3; ++r) uv[r] = sc * (-h[3 * r + a]);
    }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        if (fabs(alpha * (-h[3 * r + c]) - uv[r] * uv[c]) > 1e-12 * alpha * hmax) *bad = 1;
    ci1[q] = ci[p];
    for (int r = 0; r < 3; ++r) {
      u64[3 * q + r] = uv[r];
      if (u32) u32[3 * q + r] = (float)uv[r];
    }
    ++q;
  }
}

}  // namespace

template <typename T>
void dispatch_r1(int cpl, int variant, const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z,
                 T *Y, T alpha, T beta, T g0, T g1, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {  // shape 10: the neighbour rows of a tile staged in shared memory
    if (variant == 3 && mode != MODE_ADJ && r1_tiled_usable(A) && ld % 4 == 0 &&
        (reinterpret_cast<uintptr_t>(X) & 15) == 0) {  // 16-byte cp.async pieces
      launch_r1_tiled(A, mode, k, ld, X, W, Z, Y, nullptr, nullptr, alpha, beta, g0, g1, s);
      return;
    }
  }
  if (cpl == 4)
    dispatch_r1_variant<T, (sizeof(T) == 4 ? 4 : 2)>(variant, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
  else if (cpl == 2)
    dispatch_r1_variant<T, 2>(variant, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
  else
    dispatch_r1_variant<T, 1>(variant, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
}
template void dispatch_r1<double>(int, int, const Bsr<double> &, int, int32_t, int64_t, const double *, const double *,
                                  double *, double *, double, double, double, double, cudaStream_t);
template void dispatch_r1<float>(int, int, const Bsr<float> &, int, int32_t, int64_t, const float *, const float *,
                                 float *, float *, float, float, float, float, cudaStream_t);

void launch_build_r1(int32_t n_atoms, const int32_t *rp, const int32_t *ci, const double *H, double alpha, double shift,
                     int32_t *rp1, int32_t *ci1, double *u64, double *dg64, float *u32, float *dg32, int32_t *bad,
                     cudaStream_t s) {
  if (n_atoms <= 0) return;
  PFE_LAUNCH k_build_r1<<<(unsigned)((n_atoms + 127) / 128), 128, 0, s>>>(n_atoms, rp, ci, H, alpha, shift, rp1, ci1,
                                                                          u64, dg64, u32, dg32, bad);
}

}  // namespace pfe
