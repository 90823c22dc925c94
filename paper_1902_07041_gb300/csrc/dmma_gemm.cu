// FP64 tensor-core products of the subspace iteration (Gram matrices of CholQR2, the
// Rayleigh-Ritz projection X^T W, the projections against locked vectors, and the block
// updates X Q, X R^{-1}, Y - L h).  They are dense contractions, so they run on the FP64
// tensor pipe through mma.sync.m8n8k4.f64 (DMMA): GB300 has no FP64 form of tcgen05.  Measured,
// real DMMA GEMMs on GB300 (these kernels and cuBLAS's) reach about the FP64 FMA ceiling.
//
// Fragment layout of m8n8k4.f64 (row.col): with g = lane / 4, t = lane % 4,
//   A (8x4):  a = A[g][t];   B (4x8): b = B[t][g];   C/D (8x8): c0 = C[g][2t], c1 = C[g][2t+1].
// CTA tile 64 x 64, four warps in a 2 x 2 arrangement, each warp 32 x 32 = 4 x 4 mma tiles.
// Shared-memory rows are padded to 4 mod 16 doubles so that the fragment reads of a half warp
// hit 16 distinct 8-byte banks.
#include "pfe_internal.h"

namespace pfe {
namespace {

constexpr int TM = 64, TN = 64, KC = 16;
constexpr int LDS_G = TM + 4;  // gram: [k][64 + 4]
constexpr int LDS_U = KC + 4;  // update: [64][16 + 4]

__device__ __forceinline__ void dmma(double &c0, double &c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// Partial Gram tiles: work[z][q][p] = sum_{i in chunk z} A[i, p] B[i, q]
// (A: K x m row-major lda, B: K x nn row-major ldb).  With sym, only tiles with p-tile <= q-tile.
__global__ void __launch_bounds__(128) k_gram_partial(int64_t K, int32_t m, int32_t nn, const double *__restrict__ A,
                                                      int64_t lda, const double *__restrict__ B, int64_t ldb,
                                                      int64_t chunk, int sym, double *__restrict__ work) {
  const int tp = blockIdx.x, tq = blockIdx.y, z = blockIdx.z;
  if (sym && tp > tq) return;
  __shared__ double As[KC][LDS_G];
  __shared__ double Bs[KC][LDS_G];
  const int p0 = tp * TM, q0 = tq * TN;
  const int64_t i_begin = (int64_t)z * chunk, i_end = min(K, i_begin + chunk);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int wp = (warp >> 1) * 32, wq = (warp & 1) * 32;
  double acc[4][4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
  for (int64_t i0 = i_begin; i0 < i_end; i0 += KC) {
    for (int idx = threadIdx.x; idx < KC * TM; idx += 128) {
      const int r = idx / TM, c = idx % TM;
      const int64_t i = i0 + r;
      const bool ok = i < i_end;
      As[r][c] = (ok && p0 + c < m) ? A[i * lda + p0 + c] : 0.0;
      Bs[r][c] = (ok && q0 + c < nn) ? B[i * ldb + q0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) af[a] = As[kk + t][wp + 8 * a + g];
#pragma unroll
      for (int b = 0; b < 4; ++b) bf[b] = Bs[kk + t][wq + 8 * b + g];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dmma(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
    }
    __syncthreads();
  }
  double *wz = work + (int64_t)z * m * nn;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int p = p0 + wp + 8 * a + g;
      const int q = q0 + wq + 8 * b + 2 * t;
      if (p < m && q < nn) wz[(int64_t)q * m + p] = acc[a][b][0];
      if (p < m && q + 1 < nn) wz[(int64_t)(q + 1) * m + p] = acc[a][b][1];
    }
}

// C[q * ldc + p] = alpha * sum_z work[z][q][p] + beta * C (fixed summation order); with sym the
// lower triangle is mirrored from the upper one.
__global__ void k_gram_reduce(int32_t m, int32_t nn, int32_t splits, const double *__restrict__ work, double alpha,
                              double beta, double *C, int64_t ldc, int sym) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * nn) return;
  int32_t q = (int32_t)(t / m), p = (int32_t)(t - (int64_t)q * m);
  int32_t sp = p, sq = q;
  if (sym && (p / TM) > (q / TN)) {  // tile not computed: take the transposed entry
    sp = q;
    sq = p;
  }
  double s = 0.0;
  for (int32_t z = 0; z < splits; ++z) s += work[(int64_t)z * m * nn + (int64_t)sq * m + sp];
  const double old = (beta == 0.0) ? 0.0 : beta * C[(int64_t)q * ldc + p];
  C[(int64_t)q * ldc + p] = alpha * s + old;
}

// C (M x N row-major, ldc) = alpha * A (M x K row-major, lda) * Bc (K x N column-major, ldb) + beta * C.
// C must not overlap A.  upper: Bc is upper triangular (Bc[k][q] = 0 for k > q), so a column tile
// [q0, q0 + 64) only needs k < q0 + 64.
__global__ void __launch_bounds__(128) k_update(int64_t M, int32_t N, int32_t K, const double *__restrict__ A,
                                                int64_t lda, const double *__restrict__ Bc, int64_t ldb, double alpha,
                                                double beta, double *C, int64_t ldc, int upper) {
  const int tq = blockIdx.x;  // column tile fastest: CTAs sharing the same rows of A run together (L2 reuse)
  const int64_t ti = blockIdx.y;
  __shared__ double As[TM][LDS_U];
  __shared__ double Bs[TN][LDS_U];
  const int64_t i0 = ti * TM;
  const int q0 = tq * TN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int wi = (warp >> 1) * 32, wq = (warp & 1) * 32;
  double acc[4][4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;
  const int kend = upper ? min(K, q0 + TN) : K;
  for (int k0 = 0; k0 < kend; k0 += KC) {
    for (int idx = threadIdx.x; idx < TM * KC; idx += 128) {
      const int r = idx / KC, c = idx % KC;
      const int64_t i = i0 + r;
      const int kk = k0 + c;
      As[r][c] = (i < M && kk < K) ? A[i * lda + kk] : 0.0;
      const int q = q0 + r;
      Bs[r][c] = (q < N && kk < K) ? Bc[(int64_t)q * ldb + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) af[a] = As[wi + 8 * a + g][kk + t];
#pragma unroll
      for (int b = 0; b < 4; ++b) bf[b] = Bs[wq + 8 * b + g][kk + t];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dmma(acc[a][b][0], acc[a][b][1], af[a], bf[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t i = i0 + wi + 8 * a + g;
      const int q = q0 + wq + 8 * b + 2 * t;
      if (i >= M) continue;
      double *c = C + i * ldc;
      if (q < N) c[q] = alpha * acc[a][b][0] + (beta == 0.0 ? 0.0 : beta * c[q]);
      if (q + 1 < N) c[q + 1] = alpha * acc[a][b][1] + (beta == 0.0 ? 0.0 : beta * c[q + 1]);
    }
}

}  // namespace

int32_t gram_splits(int64_t K, int32_t m, int32_t nn, bool sym) {
  const int64_t tp = (m + TM - 1) / TM, tq = (nn + TN - 1) / TN;
  const int64_t tiles = sym ? tp * (tp + 1) / 2 : tp * tq;
  int64_t s = (8 * 152 + tiles - 1) / std::max<int64_t>(tiles, 1);
  s = std::min<int64_t>(s, std::max<int64_t>(1, K / 512));
  return (int32_t)std::max<int64_t>(1, std::min<int64_t>(s, 256));
}

size_t gram_work(int64_t K, int32_t m, int32_t nn, bool sym) {
  return (size_t)gram_splits(K, m, nn, sym) * (size_t)m * (size_t)nn;
}

void launch_gram(int64_t K, int32_t m, int32_t nn, const double *A, int64_t lda, const double *B, int64_t ldb,
                 double alpha, double beta, double *C, int64_t ldc, bool sym, double *work, cudaStream_t s) {
  if (m <= 0 || nn <= 0) return;
  const int32_t splits = gram_splits(K, m, nn, sym);
  const int64_t chunk = std::max<int64_t>(KC, ((K + splits - 1) / splits + KC - 1) / KC * KC);
  dim3 grid((m + TM - 1) / TM, (nn + TN - 1) / TN, splits);
  PFE_LAUNCH k_gram_partial<<<grid, 128, 0, s>>>(K, m, nn, A, lda, B, ldb, chunk, sym ? 1 : 0, work);
  const int64_t tot = (int64_t)m * nn;
  PFE_LAUNCH k_gram_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(m, nn, splits, work, alpha, beta, C, ldc,
                                                                         sym ? 1 : 0);
}

void launch_update(int64_t M, int32_t N, int32_t K, const double *A, int64_t lda, const double *Bc, int64_t ldb,
                   double alpha, double beta, double *C, int64_t ldc, cudaStream_t s, bool upper) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + TN - 1) / TN, (unsigned)((M + TM - 1) / TM));
  PFE_LAUNCH k_update<<<grid, 128, 0, s>>>(M, N, K, A, lda, Bc, ldb, alpha, beta, C, ldc, upper ? 1 : 0);
}

}  // namespace pfe
