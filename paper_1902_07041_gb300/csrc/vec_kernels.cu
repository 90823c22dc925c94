// Dense multivector kernels around the filter: random start blocks (Philox4x32-10),
// deterministic column reductions (norms, dots, residual norms), column scaling and
// gathers for locking, precision conversions and layout transposes for the C ABI.
// Multivectors are row-major n x k with row stride ld unless a name says otherwise.
#include <atomic>

#include "pfe_internal.h"

namespace pfe {

namespace {
std::atomic<int64_t> g_launches{0};
}
int64_t launch_count() { return g_launches.load(); }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t dbuf_reserve(DBuf &b, size_t bytes) {
  if (bytes <= b.bytes && b.p) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  else b.p = nullptr;
  return e;
}

void dbuf_free(DBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

namespace {

constexpr int kRowsPerBlock = 512;

// Philox4x32-10 of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of the two
// multiply-xor S-boxes with the Weyl key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = 0xD2511F53u * x0, hi_a = __umulhi(0xD2511F53u, x0);
    const uint32_t lo_b = 0xCD9E8D57u * x2, hi_b = __umulhi(0xCD9E8D57u, x2);
    const uint32_t y0 = hi_b ^ x1 ^ k0, y2 = hi_a ^ x3 ^ k1;
    x0 = y0;
    x1 = lo_b;
    x2 = y2;
    x3 = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Standard normal for (row, col, stream) under seed: counter (row, col, stream, 0),
// key (low, high word of seed); Box-Muller on two 53-bit uniforms, u1 in (0, 1].
__device__ double philox_normal(uint64_t seed, uint32_t stream, uint32_t row, uint32_t col) {
  uint32_t x0 = row, x1 = col, x2 = stream, x3 = 0u;
  philox4x32_10(x0, x1, x2, x3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t ua = ((uint64_t)x0 << 21) ^ (uint64_t)(x1 >> 11);
  const uint64_t ub = ((uint64_t)x2 << 21) ^ (uint64_t)(x3 >> 11);
  const double u1 = ((double)ua + 1.0) * 0x1.0p-53, u2 = (double)ub * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

template <typename T>
__global__ void k_fill_normal(uint64_t seed, uint32_t stream, int64_t n, int32_t k, int32_t col0, T *X, int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int32_t c = (int32_t)(t - i * k);
  X[i * ld + c] = (T)philox_normal(seed, stream, (uint32_t)i, (uint32_t)(col0 + c));
}

template <typename T>
__global__ void k_col_dots_partial(int64_t n, int32_t k, const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y,
                                   int64_t ldy, double *work) {
  const int32_t c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
  const int64_t r1 = min(n, r0 + kRowsPerBlock);
  double s = 0.0;
  for (int64_t i = r0; i < r1; ++i) s += (double)X[i * ldx + c] * (double)Y[i * ldy + c];
  work[(int64_t)blockIdx.x * k + c] = s;
}

__global__ void k_col_resid_partial(int64_t n, int32_t k, const double *__restrict__ W, const double *__restrict__ X,
                                    int64_t ld, const double *__restrict__ theta, double *work) {
  const int32_t c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
  const int64_t r1 = min(n, r0 + kRowsPerBlock);
  const double th = theta[c];
  double s = 0.0;
  for (int64_t i = r0; i < r1; ++i) {
    const double e = W[i * ld + c] - th * X[i * ld + c];
    s += e * e;
  }
  work[(int64_t)blockIdx.x * k + c] = s;
}

__global__ void k_col_finish(int32_t nblk, int32_t k, const double *__restrict__ work, double *out) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double s = 0.0;
  for (int32_t b = 0; b < nblk; ++b) s += work[(int64_t)b * k + c];
  out[c] = s;
}

template <typename T>
__global__ void k_scale_cols(int64_t n, int32_t k, T *X, int64_t ld, const double *__restrict__ scale) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int32_t c = (int32_t)(t - i * k);
  X[i * ld + c] = (T)((double)X[i * ld + c] * scale[c]);
}

template <typename T>
__global__ void k_axpby(int64_t n, int32_t k, T alpha, const T *__restrict__ X, int64_t ldx, T beta, T *Y,
                        int64_t ldy) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int32_t c = (int32_t)(t - i * k);
  const T y = (beta == T(0)) ? T(0) : beta * Y[i * ldy + c];
  Y[i * ldy + c] = alpha * X[i * ldx + c] + y;
}

template <typename Tin, typename Tout>
__global__ void k_convert(int64_t n, int32_t k, const Tin *__restrict__ X, int64_t ldx, Tout *Y, int64_t ldy) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int32_t c = (int32_t)(t - i * k);
  Y[i * ldy + c] = (Tout)X[i * ldx + c];
}

__global__ void k_gather_cols(int64_t n, int32_t kd, const double *__restrict__ src, int64_t lds, double *dst,
                              int64_t ldd, const int32_t *__restrict__ idx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * kd) return;
  const int64_t i = t / kd;
  const int32_t c = (int32_t)(t - i * kd);
  dst[i * ldd + c] = src[i * lds + idx[c]];
}

// tiled transposes through shared memory: (rows of n) x (cols of k)
template <typename T>
__global__ void k_col_to_row(int64_t n, int32_t k, const T *__restrict__ C, int64_t ldc, T *R, int64_t ldr) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int32_t c0 = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {  // read: consecutive i along threadIdx.x
    const int32_t c = c0 + yy;
    const int64_t i = i0 + threadIdx.x;
    if (c < k && i < n) tile[yy][threadIdx.x] = C[(int64_t)c * ldc + i];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {  // write: consecutive c along threadIdx.x
    const int64_t i = i0 + yy;
    const int32_t c = c0 + threadIdx.x;
    if (c < k && i < n) R[i * ldr + c] = tile[threadIdx.x][yy];
  }
}

template <typename T>
__global__ void k_row_to_col(int64_t n, int32_t k, const T *__restrict__ R, int64_t ldr, T *C, int64_t ldc) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int32_t c0 = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t i = i0 + yy;
    const int32_t c = c0 + threadIdx.x;
    if (c < k && i < n) tile[yy][threadIdx.x] = R[i * ldr + c];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int32_t c = c0 + yy;
    const int64_t i = i0 + threadIdx.x;
    if (c < k && i < n) C[(int64_t)c * ldc + i] = tile[threadIdx.x][yy];
  }
}

inline unsigned grid1(int64_t total, int threads = 256) { return (unsigned)((total + threads - 1) / threads); }

// out = max_ij |G_ij - delta_ij| over a k x k matrix, one block
__global__ void k_max_dev_identity(int32_t k, const double *__restrict__ G, double *out) {
  __shared__ double red[1024];
  double m = 0.0;
  const int64_t tot = (int64_t)k * k;
  for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
    const int64_t i = t / k, j = t - i * k;
    m = fmax(m, fabs(G[t] - (i == j ? 1.0 : 0.0)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

void launch_max_dev_identity(int32_t k, const double *G, double *out, cudaStream_t s) {
  PFE_LAUNCH k_max_dev_identity<<<1, 1024, 0, s>>>(k, G, out);
}

template <typename T>
void launch_fill_normal(uint64_t seed, uint32_t stream_id, int64_t n, int32_t k, int32_t col0, T *X, int64_t ld,
                        cudaStream_t s) {
  if (n <= 0 || k <= 0) return;
  PFE_LAUNCH k_fill_normal<T><<<grid1(n * k), 256, 0, s>>>(seed, stream_id, n, k, col0, X, ld);
}
template void launch_fill_normal<double>(uint64_t, uint32_t, int64_t, int32_t, int32_t, double *, int64_t, cudaStream_t);
template void launch_fill_normal<float>(uint64_t, uint32_t, int64_t, int32_t, int32_t, float *, int64_t, cudaStream_t);

size_t colreduce_work(int64_t n, int32_t k) {
  const int64_t nblk = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  return (size_t)(nblk > 0 ? nblk : 1) * (size_t)(k > 0 ? k : 1);
}

template <typename T>
void launch_col_dots(int64_t n, int32_t k, const T *X, int64_t ldx, const T *Y, int64_t ldy, double *out, double *work,
                     cudaStream_t s) {
  if (k <= 0) return;
  const int32_t nblk = (int32_t)((n + kRowsPerBlock - 1) / kRowsPerBlock);
  if (nblk > 0) {
    dim3 g(nblk, (k + 255) / 256);
    PFE_LAUNCH k_col_dots_partial<T><<<g, 256, 0, s>>>(n, k, X, ldx, Y, ldy, work);
  }
  PFE_LAUNCH k_col_finish<<<grid1(k), 256, 0, s>>>(nblk, k, work, out);
}
template void launch_col_dots<double>(int64_t, int32_t, const double *, int64_t, const double *, int64_t, double *,
                                      double *, cudaStream_t);
template void launch_col_dots<float>(int64_t, int32_t, const float *, int64_t, const float *, int64_t, double *,
                                     double *, cudaStream_t);

void launch_col_resid2(int64_t n, int32_t k, const double *W, const double *X, int64_t ld, const double *theta,
                       double *out, double *work, cudaStream_t s) {
  if (k <= 0) return;
  const int32_t nblk = (int32_t)((n + kRowsPerBlock - 1) / kRowsPerBlock);
  if (nblk > 0) {
    dim3 g(nblk, (k + 255) / 256);
    PFE_LAUNCH k_col_resid_partial<<<g, 256, 0, s>>>(n, k, W, X, ld, theta, work);
  }
  PFE_LAUNCH k_col_finish<<<grid1(k), 256, 0, s>>>(nblk, k, work, out);
}

template <typename T>
void launch_scale_cols(int64_t n, int32_t k, T *X, int64_t ld, const double *scale, cudaStream_t s) {
  if (n <= 0 || k <= 0) return;
  PFE_LAUNCH k_scale_cols<T><<<grid1(n * k), 256, 0, s>>>(n, k, X, ld, scale);
}
template void launch_scale_cols<double>(int64_t, int32_t, double *, int64_t, const double *, cudaStream_t);
template void launch_scale_cols<float>(int64_t, int32_t, float *, int64_t, const double *, cudaStream_t);

template <typename T>
void launch_axpby(int64_t n, int32_t k, T alpha, const T *X, int64_t ldx, T beta, T *Y, int64_t ldy, cudaStream_t s) {
  if (n <= 0 || k <= 0) return;
  PFE_LAUNCH k_axpby<T><<<grid1(n * k), 256, 0, s>>>(n, k, alpha, X, ldx, beta, Y, ldy);
}
template void launch_axpby<double>(int64_t, int32_t, double, const double *, int64_t, double, double *, int64_t,
                                   cudaStream_t);
template void launch_axpby<float>(int64_t, int32_t, float, const float *, int64_t, float, float *, int64_t,
                                  cudaStream_t);

template <typename Tin, typename Tout>
void launch_convert(int64_t n, int32_t k, const Tin *X, int64_t ldx, Tout *Y, int64_t ldy, cudaStream_t s) {
  if (n <= 0 || k <= 0) return;
  PFE_LAUNCH k_convert<Tin, Tout><<<grid1(n * k), 256, 0, s>>>(n, k, X, ldx, Y, ldy);
}
template void launch_convert<double, float>(int64_t, int32_t, const double *, int64_t, float *, int64_t, cudaStream_t);
template void launch_convert<float, double>(int64_t, int32_t, const float *, int64_t, double *, int64_t, cudaStream_t);

void launch_gather_cols(int64_t n, int32_t kdst, const double *src, int64_t lds, double *dst, int64_t ldd,
                        const int32_t *idx, cudaStream_t s) {
  if (n <= 0 || kdst <= 0) return;
  PFE_LAUNCH k_gather_cols<<<grid1(n * kdst), 256, 0, s>>>(n, kdst, src, lds, dst, ldd, idx);
}

template <typename T>
void launch_colmajor_to_rowmajor(int64_t n, int32_t k, const T *C, int64_t ldc, T *R, int64_t ldr, cudaStream_t s) {
  if (n <= 0 || k <= 0) return;
  dim3 g((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
  PFE_LAUNCH k_col_to_row<T><<<g, dim3(32, 8), 0, s>>>(n, k, C, ldc, R, ldr);
}
template <typename T>
void launch_rowmajor_to_colmajor(int64_t n, int32_t k, const T *R, int64_t ldr, T *C, int64_t ldc, cudaStream_t s) {
  if (n <= 0 || k <= 0) return;
  dim3 g((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
  PFE_LAUNCH k_row_to_col<T><<<g, dim3(32, 8), 0, s>>>(n, k, R, ldr, C, ldc);
}
template void launch_colmajor_to_rowmajor<double>(int64_t, int32_t, const double *, int64_t, double *, int64_t,
                                                  cudaStream_t);
template void launch_colmajor_to_rowmajor<float>(int64_t, int32_t, const float *, int64_t, float *, int64_t,
                                                 cudaStream_t);
template void launch_rowmajor_to_colmajor<double>(int64_t, int32_t, const double *, int64_t, double *, int64_t,
                                                  cudaStream_t);
template void launch_rowmajor_to_colmajor<float>(int64_t, int32_t, const float *, int64_t, float *, int64_t,
                                                 cudaStream_t);

template <typename T>
void launch_zero(T *p, int64_t count, cudaStream_t s) {
  if (count > 0) cudaMemsetAsync(p, 0, sizeof(T) * (size_t)count, s);
}
template void launch_zero<double>(double *, int64_t, cudaStream_t);
template void launch_zero<float>(float *, int64_t, cudaStream_t);

}  // namespace pfe
