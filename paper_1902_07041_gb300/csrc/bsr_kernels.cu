// BSR kernels of the filter: the fused Chebyshev step of Alg. 2 over 3x3 blocks, the mass
// weighting of eq. (2), the scaled filter operator of eq. (transf.1), and the adjoint's
// outer products and chain rule.
//
// Multivector layout: row-major n x k with row stride ld (the k columns of one dof row are
// contiguous).  The three dof rows of atom j are then 3k contiguous values, so gathering a
// neighbour's rows is one coalesced sweep per row.  One warp owns (atom i, a chunk of
// 32 * CPL columns); each lane owns CPL adjacent columns and keeps 3 x CPL accumulators.
// Block values and column indices are warp-uniform loads (served as L1 broadcasts); every
// 3x3 block is read once per column chunk.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "pfe_internal.h"
#include "vec_io.cuh"

namespace pfe {
namespace {

// ---- the fused step -------------------------------------------------------------------
// SPMM : Z = alpha A X
// FIRST: Z = alpha A X;          Y = g0 X + g1 Z            (t_1 and p_1(H)x of Alg. 2)
// STEP : Z = alpha A X + beta W; Y += g1 Z if Y            (t_{j+1} = 2 Ht t_j - t_{j-1})
// STEP_ACC: as STEP with Y += g0 X + g1 Z                   (the term of t_j added one step late, so
//        that y is read and written every other step)
// ADJ  : Z = alpha A X + beta W + g0 Y   (Y read-only)      (reverse sweep of the adjoint)
// With A = (2/d)(H - cI) the step needs alpha = 1, beta = -1; the first step alpha = 1/2.
// GROUPED: the 8 warps of a CTA take 8 consecutive atoms of one column chunk (their neighbour
// rows overlap, so gathers hit L1); otherwise a warp takes (atom, chunk) with chunk fastest.
// UNROLL = 2: two blocks per iteration, so six row gathers are in flight per lane.
template <typename T, int CPL, int MODE, bool GROUPED, int UNROLL, int MINB = 1>
__global__ void __launch_bounds__(256, MINB) k_bsr_step(int32_t n_atoms, const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ ci, const T *__restrict__ vals,
                                                  int32_t k, int64_t ld, int32_t nchunk, const T *__restrict__ X,
                                                  const T *W, T *Z, T *Y, T alpha, T beta, T g0, T g1) {
  const int lane = threadIdx.x & 31;
  int64_t atom;
  int chunk;
  if (GROUPED) {
    const int64_t b = blockIdx.x;
    chunk = (int)(b % nchunk);
    atom = (b / nchunk) * 8 + (threadIdx.x >> 5);
  } else {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    atom = gw / nchunk;
    chunk = (int)(gw - atom * nchunk);
  }
  if (atom >= n_atoms) return;
  const int c0 = (chunk * 32 + lane) * CPL;
  const bool on = c0 < k;
  T acc[3][CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) acc[0][c] = acc[1][c] = acc[2][c] = T(0);
  const int p0 = __ldg(rp + atom), p1 = __ldg(rp + atom + 1);
  for (int p = p0; p < p1; p += UNROLL) {
    T a[UNROLL][9];
    T x[UNROLL][3][CPL];
    bool has[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      has[u] = (p + u) < p1;
      const int pu = has[u] ? p + u : p;
      const int64_t j = __ldg(ci + pu);
      const T *v = vals + 9 * (int64_t)pu;
#pragma unroll
      for (int t = 0; t < 9; ++t) a[u][t] = __ldg(v + t);
      if (on) {
        const T *xr = X + 3 * j * ld + c0;
        ldg_n(xr, x[u][0]);
        ldg_n(xr + ld, x[u][1]);
        ldg_n(xr + 2 * ld, x[u][2]);
      }
    }
    if (on) {
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        if (!has[u]) continue;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          acc[0][c] = fma(a[u][0], x[u][0][c], fma(a[u][1], x[u][1][c], fma(a[u][2], x[u][2][c], acc[0][c])));
          acc[1][c] = fma(a[u][3], x[u][0][c], fma(a[u][4], x[u][1][c], fma(a[u][5], x[u][2][c], acc[1][c])));
          acc[2][c] = fma(a[u][6], x[u][0][c], fma(a[u][7], x[u][1][c], fma(a[u][8], x[u][2][c], acc[2][c])));
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
      T xo[CPL], y[CPL];
      ldg_n(X + off, xo);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g1, z[c], g0 * xo[c]);
      st_n(Y + off, y);
    } else if (MODE == MODE_STEP && Y != nullptr) {
      T y[CPL];
      ld_n(Y + off, y);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g1, z[c], y[c]);
      st_n(Y + off, y);
    } else if (MODE == MODE_STEP_ACC) {  // also the pending term g0 t_j (this atom's rows of X)
      T y[CPL], xo[CPL];
      ld_n(Y + off, y);
      ldg_n(X + off, xo);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g0, xo[c], fma(g1, z[c], y[c]));
      st_n(Y + off, y);
    }
  }
}

// Shape 4: the neighbour rows are staged in shared memory by asynchronous copies (cp.async),
// STAGES blocks ahead of the FMAs, in a ring private to each warp.  Each lane copies and later
// reads only its own 16 bytes of every row, so no warp-level barrier is needed; the copies keep
// STAGES x 3 row gathers in flight per warp without holding registers.  Needs 16-byte lanes
// (float x 4 or double x 2).
constexpr int kStages = 4;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <typename T, int CPL, int MODE>
__global__ void __launch_bounds__(256) k_bsr_step_async(int32_t n_atoms, const int32_t *__restrict__ rp,
                                                        const int32_t *__restrict__ ci, const T *__restrict__ vals,
                                                        int32_t k, int64_t ld, int32_t nchunk, const T *__restrict__ X,
                                                        const T *W, T *Z, T *Y, T alpha, T beta, T g0, T g1) {
  static_assert(sizeof(T) * CPL == 16, "16-byte lanes");
  __shared__ __align__(16) T ring[8][kStages][3][32 * CPL];  // [warp][stage][row][lane * CPL]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t atom = gw / nchunk;
  if (atom >= n_atoms) return;
  const int chunk = (int)(gw - atom * nchunk);
  const int c0 = (chunk * 32 + lane) * CPL;
  const bool on = c0 < k;
  T acc[3][CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) acc[0][c] = acc[1][c] = acc[2][c] = T(0);
  const int p0 = __ldg(rp + atom), nb = __ldg(rp + atom + 1) - p0;
  auto issue = [&](int b) {
    if (b < nb && on) {
      const int64_t j = __ldg(ci + p0 + b);
      const T *xr = X + 3 * j * ld + c0;
      T *dst = &ring[warp][b % kStages][0][lane * CPL];
      cp_async16(dst, xr);
      cp_async16(dst + 32 * CPL, xr + ld);
      cp_async16(dst + 64 * CPL, xr + 2 * ld);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int b = 0; b < kStages - 1; ++b) issue(b);
  for (int b = 0; b < nb; ++b) {
    issue(b + kStages - 1);
    cp_async_wait<kStages - 1>();
    const T *v = vals + 9 * (int64_t)(p0 + b);
    T a[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) a[t] = __ldg(v + t);
    if (on) {
      const T *src = &ring[warp][b % kStages][0][lane * CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const T x0 = src[c], x1 = src[32 * CPL + c], x2 = src[64 * CPL + c];
        acc[0][c] = fma(a[0], x0, fma(a[1], x1, fma(a[2], x2, acc[0][c])));
        acc[1][c] = fma(a[3], x0, fma(a[4], x1, fma(a[5], x2, acc[1][c])));
        acc[2][c] = fma(a[6], x0, fma(a[7], x1, fma(a[8], x2, acc[2][c])));
      }
    }
  }
  cp_async_wait<0>();
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
      T xo[CPL], y[CPL];
      ldg_n(X + off, xo);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g1, z[c], g0 * xo[c]);
      st_n(Y + off, y);
    } else if (MODE == MODE_STEP && Y != nullptr) {
      T y[CPL];
      ld_n(Y + off, y);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g1, z[c], y[c]);
      st_n(Y + off, y);
    } else if (MODE == MODE_STEP_ACC) {  // also the pending term g0 t_j (this atom's rows of X)
      T y[CPL], xo[CPL];
      ld_n(Y + off, y);
      ldg_n(X + off, xo);
#pragma unroll
      for (int c = 0; c < CPL; ++c) y[c] = fma(g0, xo[c], fma(g1, z[c], y[c]));
      st_n(Y + off, y);
    }
  }
}

template <typename T, int CPL>
void dispatch_async(const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z, T *Y, T alpha,
                    T beta, T g0, T g1, cudaStream_t s) {
  const int32_t nchunk = (k + 32 * CPL - 1) / (32 * CPL);
  const int64_t blocks = ((int64_t)A.n_atoms * nchunk * 32 + 255) / 256;
#define PFE_ASYNC_LAUNCH(M)                                                                                 \
  PFE_LAUNCH k_bsr_step_async<T, CPL, M><<<(unsigned)blocks, 256, 0, s>>>(A.n_atoms, A.rp, A.ci, A.vals, k, ld, \
                                                                           nchunk, X, W, Z, Y, alpha, beta, g0, g1)
  if (mode == MODE_SPMM)
    PFE_ASYNC_LAUNCH(MODE_SPMM);
  else if (mode == MODE_FIRST)
    PFE_ASYNC_LAUNCH(MODE_FIRST);
  else if (mode == MODE_ADJ)
    PFE_ASYNC_LAUNCH(MODE_ADJ);
  else if (mode == MODE_STEP_ACC)
    PFE_ASYNC_LAUNCH(MODE_STEP_ACC);
  else
    PFE_ASYNC_LAUNCH(MODE_STEP);
#undef PFE_ASYNC_LAUNCH
}

template <typename T, int CPL, bool GROUPED, int UNROLL, int MINB = 1>
void dispatch_mode(const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z, T *Y, T alpha,
                   T beta, T g0, T g1, cudaStream_t s) {
  const int32_t nchunk = (k + 32 * CPL - 1) / (32 * CPL);
  const int64_t blocks = GROUPED ? ((int64_t)A.n_atoms + 7) / 8 * nchunk
                                 : ((int64_t)A.n_atoms * nchunk * 32 + 255) / 256;
#define PFE_STEP_LAUNCH(M)                                                                                 \
  PFE_LAUNCH k_bsr_step<T, CPL, M, GROUPED, UNROLL, MINB><<<(unsigned)blocks, 256, 0, s>>>(               \
      A.n_atoms, A.rp, A.ci, A.vals, k, ld, nchunk, X, W, Z, Y, alpha, beta, g0, g1)
  if (mode == MODE_SPMM)
    PFE_STEP_LAUNCH(MODE_SPMM);
  else if (mode == MODE_FIRST)
    PFE_STEP_LAUNCH(MODE_FIRST);
  else if (mode == MODE_ADJ)
    PFE_STEP_LAUNCH(MODE_ADJ);
  else if (mode == MODE_STEP_ACC)
    PFE_STEP_LAUNCH(MODE_STEP_ACC);
  else
    PFE_STEP_LAUNCH(MODE_STEP);
#undef PFE_STEP_LAUNCH
}

template <typename T, int CPL>
void dispatch_variant(int variant, const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z,
                      T *Y, T alpha, T beta, T g0, T g1, cudaStream_t s) {
  switch (variant) {
    case 1: dispatch_mode<T, CPL, true, 1>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
    case 2: dispatch_mode<T, CPL, false, 2>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
    case 3: dispatch_mode<T, CPL, true, 2>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
    case 5: dispatch_mode<T, CPL, false, 1, 5>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
    case 6: dispatch_mode<T, CPL, true, 1, 5>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
    case 4:
      if constexpr (sizeof(T) * CPL == 16)
        dispatch_async<T, CPL>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
      else
        dispatch_mode<T, CPL, false, 1>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
      break;
    default: dispatch_mode<T, CPL, false, 1>(A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s); break;
  }
}

bool aligned(const void *p, size_t a) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

// Kernel shape of the fused step: 0 = warp per (atom, chunk), 1 = CTA per 8 atoms x chunk,
// 2 = as 0 with two blocks in flight, 3 = as 1 with two blocks in flight, 4 = rows staged in
// shared memory by cp.async, four blocks ahead (16-byte lanes only; else shape 0), 5 and 6 = as
// 0 and 1 compiled for five resident CTAs per SM (at most 51 registers a thread).  Shapes 7, 8, 9
// run on the rank-1 form of the operator when it has one (r1_kernels.cu: warp per (atom, chunk);
// five resident CTAs; two blocks in flight); without it they fall back to shape 0.
// A forced shape (set_step_variant) wins; otherwise the autotuner's choice for (type, columns per
// lane, column chunks, rank-1 form present) is used, and the default 0 before any tuning.
namespace {
// The tuner times the full-block shapes 0-6, or the rank-1 shapes 7-9 when the operator has that form.
// Shape 10 (FP32, rows staged in shared memory) runs only when forced: it measured 3.6x slower than
// shape 8 (its load phase leaves 24 warps per SM waiting, where the gathers of shape 8 overlap).
constexpr int kVariants = 7, kStagedVariant = 10, kSixCtaVariant = 11;
constexpr int kR1Candidates[] = {7, 8, 9, 11};  // rank-1 shapes the tuner times (11: as 8 at six CTAs per SM)
int g_forced[2] = {-1, -1};  // [double, float]
std::mutex g_tune_mu;
std::mutex g_tune_run_mu;
std::map<std::tuple<int, int, int, int>, int> g_tuned;  // (is_float, CPL, min(nchunk, 16), rank-1) -> shape

int pick_variant(int is_float, int cpl, int32_t nchunk, bool r1) {
  if (g_forced[is_float] >= 0) return g_forced[is_float];
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple(is_float, cpl, std::min(nchunk, 16), r1 ? 1 : 0));
  return it == g_tuned.end() ? 0 : it->second;
}
}  // namespace

void set_step_variant(int is_float, int variant) { g_forced[is_float ? 1 : 0] = variant; }

bool step_prefers_tiled(int32_t, int64_t) { return g_forced[1] == kStagedVariant; }

bool step_prefers_six_ctas(int32_t k, int64_t ld) {
  const int cpl = (k > 64 && ld % 4 == 0) ? 4 : ((k > 32 && ld % 2 == 0) ? 2 : 1);
  return pick_variant(1, cpl, (k + 32 * cpl - 1) / (32 * cpl), true) == kSixCtaVariant;
}
int step_variant(int is_float) { return g_forced[is_float ? 1 : 0]; }

namespace {
std::atomic<int> g_last_variant[2] = {{-1}, {-1}};
}
int step_last_variant(int is_float) { return g_last_variant[is_float ? 1 : 0].load(); }
void note_step_variant(int is_float, int variant) { g_last_variant[is_float ? 1 : 0].store(variant); }
void reset_step_last_variant() {
  g_last_variant[0].store(-1);
  g_last_variant[1].store(-1);
}

namespace {
template <typename T>
int cpl_for(int32_t k, int64_t ld, bool al16, bool al8);
template <>
int cpl_for<double>(int32_t k, int64_t ld, bool al16, bool) { return (k > 32 && ld % 2 == 0 && al16) ? 2 : 1; }
template <>
int cpl_for<float>(int32_t k, int64_t ld, bool al16, bool al8) {
  return (k > 64 && ld % 4 == 0 && al16) ? 4 : (k > 32 && ld % 2 == 0 && al8) ? 2 : 1;
}

template <typename T>
void dispatch_cpl(int cpl, int variant, const Bsr<T> &A, int mode, int32_t k, int64_t ld, const T *X, const T *W, T *Z,
                  T *Y, T alpha, T beta, T g0, T g1, cudaStream_t s) {
  if (variant >= kVariants) {
    if (A.u && A.dg && A.rp1 && A.ci1) {
      dispatch_r1<T>(cpl, variant - kVariants, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
      return;
    }
    variant = 0;
  }
  if (cpl == 4)
    dispatch_variant<T, (sizeof(T) == 4 ? 4 : 2)>(variant, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
  else if (cpl == 2)
    dispatch_variant<T, 2>(variant, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
  else
    dispatch_variant<T, 1>(variant, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
}
}  // namespace

// Autotuner of the step's kernel shape: times every shape as a plain product X -> scratch (the
// scratch is overwritten afterwards) and keeps the fastest for this (type, CPL, chunk count).
template <typename T>
void tune_step(const Bsr<T> &A, int32_t k, int64_t ld, const T *X, T *scratch, cudaStream_t s) {
  if (k <= 0 || A.n_atoms <= 0) return;
  const int is_float = sizeof(T) == 4;
  if (g_forced[is_float] >= 0) return;
  const int cpl = cpl_for<T>(k, ld, aligned(X, 16) && aligned(scratch, 16), aligned(X, 8) && aligned(scratch, 8));
  const int32_t nchunk = (k + 32 * cpl - 1) / (32 * cpl);
  const bool r1 = A.u != nullptr;
  const auto key = std::make_tuple(is_float, cpl, std::min(nchunk, 16), r1 ? 1 : 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tuned.count(key)) return;
  }
  // one tuning run at a time (host threads of a batched solve would otherwise time each other)
  std::lock_guard<std::mutex> run_lock(g_tune_run_mu);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tuned.count(key)) return;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  float best = 1e30f;
  int best_v = r1 ? kVariants : 0;
  std::vector<int> cands;
  if (r1)
    cands.assign(std::begin(kR1Candidates), std::end(kR1Candidates));
  else
    for (int v = 0; v < kVariants; ++v) cands.push_back(v);
  // with the rank-1 form only its shapes compete: they do a third fewer FMAs and read a third of
  // the matrix bytes of the full-block shapes
  for (int v : cands) {
    float t = 1e30f;
    for (int trial = 0; trial < 2; ++trial) {
      cudaEventRecord(e0, s);
      dispatch_cpl<T>(cpl, v, A, MODE_SPMM, k, ld, X, nullptr, scratch, nullptr, T(1), T(0), T(0), T(0), s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (trial == 1) t = ms;
    }
    if (t < best) {
      best = t;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = best_v;
}
template void tune_step<double>(const Bsr<double> &, int32_t, int64_t, const double *, double *, cudaStream_t);
template void tune_step<float>(const Bsr<float> &, int32_t, int64_t, const float *, float *, cudaStream_t);

template <>
void launch_bsr_step<double>(const Bsr<double> &A, int mode, int32_t k, int64_t ld, const double *X, const double *W,
                             double *Z, double *Y, double alpha, double beta, double g0, double g1, cudaStream_t s) {
  if (k <= 0 || A.n_atoms <= 0) return;
  const bool al16 = aligned(X, 16) && aligned(W, 16) && aligned(Z, 16) && aligned(Y, 16);
  const int cpl = cpl_for<double>(k, ld, al16, false);
  const int v = pick_variant(0, cpl, (k + 32 * cpl - 1) / (32 * cpl), A.u != nullptr);
  if (mode == MODE_FIRST || mode == MODE_STEP || mode == MODE_STEP_ACC) g_last_variant[0].store((v >= kVariants && !A.u) ? 0 : v);
  dispatch_cpl<double>(cpl, v, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
}

template <>
void launch_bsr_step<float>(const Bsr<float> &A, int mode, int32_t k, int64_t ld, const float *X, const float *W,
                            float *Z, float *Y, float alpha, float beta, float g0, float g1, cudaStream_t s) {
  if (k <= 0 || A.n_atoms <= 0) return;
  const bool al16 = aligned(X, 16) && aligned(W, 16) && aligned(Z, 16) && aligned(Y, 16);
  const bool al8 = aligned(X, 8) && aligned(W, 8) && aligned(Z, 8) && aligned(Y, 8);
  const int cpl = cpl_for<float>(k, ld, al16, al8);
  const int v = pick_variant(1, cpl, (k + 32 * cpl - 1) / (32 * cpl), A.u != nullptr);
  if (mode == MODE_FIRST || mode == MODE_STEP || mode == MODE_STEP_ACC) g_last_variant[1].store((v >= kVariants && !A.u) ? 0 : v);
  dispatch_cpl<float>(cpl, v, A, mode, k, ld, X, W, Z, Y, alpha, beta, g0, g1, s);
}

// ---- a0: mass weighting, one warp per atom row ----------------------------------------
namespace {
__global__ void k_mass_weight(int32_t n_atoms, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const double *__restrict__ delta, const double *__restrict__ mass, double *H) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n_atoms) return;
  const double mi = mass[i];
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
    const double s = sqrt(mi * mass[ci[p]]);
#pragma unroll
    for (int t = 0; t < 9; ++t) H[9 * (int64_t)p + t] = delta[9 * (int64_t)p + t] / s;
  }
}

__global__ void k_filter_matrix(int32_t n_atoms, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const double *__restrict__ H, double alpha, double shift, double *out64,
                                float *out32) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n_atoms) return;
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
    const bool diag = ci[p] == i;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const double h = H[9 * (int64_t)p + t] - ((diag && (t == 0 || t == 4 || t == 8)) ? shift : 0.0);
      const double v = alpha * h;
      if (out64) out64[9 * (int64_t)p + t] = v;
      if (out32) out32[9 * (int64_t)p + t] = (float)v;
    }
  }
}

__device__ int find_block(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t row, int32_t col) {
  int lo = rp[row], hi = rp[row + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = ci[mid];
    if (c == col) return mid;
    if (c < col) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

__device__ double rbr(const double *__restrict__ blk, const double r0, const double r1, const double r2) {
  // r^T B r for a row-major 3x3 block B
  return r0 * (blk[0] * r0 + blk[1] * r1 + blk[2] * r2) + r1 * (blk[3] * r0 + blk[4] * r1 + blk[5] * r2) +
         r2 * (blk[6] * r0 + blk[7] * r1 + blk[8] * r2);
}

__global__ void k_chain_k(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ mass,
                          int64_t nbonds, const int32_t *__restrict__ bi, const int32_t *__restrict__ bj,
                          const double *__restrict__ rhat, const double *__restrict__ hbar, double *kbar) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nbonds) return;
  const int32_t i = bi[e], j = bj[e];
  const double r0 = rhat[3 * e], r1 = rhat[3 * e + 1], r2 = rhat[3 * e + 2];
  const int pij = find_block(rp, ci, i, j), pji = find_block(rp, ci, j, i);
  const int pii = find_block(rp, ci, i, i), pjj = find_block(rp, ci, j, j);
  if (pij < 0 || pji < 0 || pii < 0 || pjj < 0) {
    kbar[e] = __longlong_as_double(0x7ff8000000000000ULL);  // NaN: bond not in the pattern
    return;
  }
  const double off = rbr(hbar + 9 * (int64_t)pij, r0, r1, r2) + rbr(hbar + 9 * (int64_t)pji, r0, r1, r2);
  kbar[e] = -off / sqrt(mass[i] * mass[j]) + rbr(hbar + 9 * (int64_t)pii, r0, r1, r2) / mass[i] +
            rbr(hbar + 9 * (int64_t)pjj, r0, r1, r2) / mass[j];
}

__global__ void k_chain_m(int32_t n_atoms, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ H, const double *__restrict__ mass,
                          const double *__restrict__ hbar, double *mbar) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_atoms) return;
  double off = 0.0, dia = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int32_t j = ci[p];
    double s = 0.0;
    for (int t = 0; t < 9; ++t) s += hbar[9 * (int64_t)p + t] * H[9 * (int64_t)p + t];
    if (j == i) {
      dia += s;
      continue;
    }
    off += s;
    const int q = find_block(rp, ci, j, (int32_t)i);
    if (q >= 0)
      for (int t = 0; t < 9; ++t) off += hbar[9 * (int64_t)q + t] * H[9 * (int64_t)q + t];
  }
  mbar[i] = -off / (2.0 * mass[i]) - dia / mass[i];
}

// Segment form of the adjoint's pattern-restricted outer products:
//   hbar[9p + 3r + s] += sum_q alpha_q sum_c A_q[3i + r, c] * T_q[3j + s, c],   block p = (i, j),
// with A_q = A0 + q * stride, T_q = T0 + q * stride (q = 0 .. nq - 1), alpha_q = alpha except
// alpha_0 = alpha0.  One group of four lanes per stored block; the lanes split the contraction over
// (q, column pairs) and meet in two shuffle steps.  The row i of block p comes from a binary search
// of row_ptr.  ld is even and A0, T0 and stride keep every row start 16-byte aligned.
__global__ void __launch_bounds__(256) k_outer_accum_seg(int32_t n_atoms, int64_t nnzb, const int32_t *__restrict__ rp,
                                                         const int32_t *__restrict__ ci, int32_t k, int64_t ld,
                                                         int32_t nq, int64_t stride, const double *__restrict__ A0,
                                                         const double *__restrict__ T0, double alpha0, double alpha,
                                                         double *__restrict__ hbar) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const int l4 = threadIdx.x & 3;
  const bool live = g < nnzb;
  const int64_t p = live ? g : nnzb - 1;
  int32_t lo = 0, hi = n_atoms;  // largest i with rp[i] <= p
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (rp[mid] <= p) lo = mid;
    else hi = mid;
  }
  const int64_t i = lo, j = ci[p];
  double s[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) s[t] = 0.0;
  for (int32_t q = 0; q < nq; ++q) {
    const double *a = A0 + q * stride + 3 * i * ld, *t = T0 + q * stride + 3 * j * ld;
    double u[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = 0.0;
    for (int32_t c = 2 * l4; c < k; c += 8) {
      if (c + 1 < k) {
        const double2 a0 = __ldg(reinterpret_cast<const double2 *>(a + c));
        const double2 a1 = __ldg(reinterpret_cast<const double2 *>(a + ld + c));
        const double2 a2 = __ldg(reinterpret_cast<const double2 *>(a + 2 * ld + c));
        const double2 t0 = __ldg(reinterpret_cast<const double2 *>(t + c));
        const double2 t1 = __ldg(reinterpret_cast<const double2 *>(t + ld + c));
        const double2 t2 = __ldg(reinterpret_cast<const double2 *>(t + 2 * ld + c));
        u[0] = fma(a0.x, t0.x, fma(a0.y, t0.y, u[0]));
        u[1] = fma(a0.x, t1.x, fma(a0.y, t1.y, u[1]));
        u[2] = fma(a0.x, t2.x, fma(a0.y, t2.y, u[2]));
        u[3] = fma(a1.x, t0.x, fma(a1.y, t0.y, u[3]));
        u[4] = fma(a1.x, t1.x, fma(a1.y, t1.y, u[4]));
        u[5] = fma(a1.x, t2.x, fma(a1.y, t2.y, u[5]));
        u[6] = fma(a2.x, t0.x, fma(a2.y, t0.y, u[6]));
        u[7] = fma(a2.x, t1.x, fma(a2.y, t1.y, u[7]));
        u[8] = fma(a2.x, t2.x, fma(a2.y, t2.y, u[8]));
      } else {
        const double a0 = a[c], a1 = a[ld + c], a2 = a[2 * ld + c];
        const double t0 = t[c], t1 = t[ld + c], t2 = t[2 * ld + c];
        u[0] = fma(a0, t0, u[0]); u[1] = fma(a0, t1, u[1]); u[2] = fma(a0, t2, u[2]);
        u[3] = fma(a1, t0, u[3]); u[4] = fma(a1, t1, u[4]); u[5] = fma(a1, t2, u[5]);
        u[6] = fma(a2, t0, u[6]); u[7] = fma(a2, t1, u[7]); u[8] = fma(a2, t2, u[8]);
      }
    }
    const double w = q == 0 ? alpha0 : alpha;
#pragma unroll
    for (int e = 0; e < 9; ++e) s[e] = fma(w, u[e], s[e]);
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    s[e] += __shfl_xor_sync(0xffffffffu, s[e], 1);
    s[e] += __shfl_xor_sync(0xffffffffu, s[e], 2);
  }
  if (live) {
#pragma unroll
    for (int e = 0; e < 9; ++e)
      if ((e & 3) == l4) hbar[9 * p + e] += s[e];
  }
}
}  // namespace

void launch_mass_weight(int32_t n_atoms, const int32_t *rp, const int32_t *ci, const double *delta, const double *mass,
                        double *H, cudaStream_t s) {
  const int64_t blocks = ((int64_t)n_atoms * 32 + 255) / 256;
  PFE_LAUNCH k_mass_weight<<<(unsigned)blocks, 256, 0, s>>>(n_atoms, rp, ci, delta, mass, H);
}

void launch_filter_matrix(int32_t n_atoms, const int32_t *rp, const int32_t *ci, const double *H, double alpha,
                          double shift, double *out64, float *out32, cudaStream_t s) {
  const int64_t blocks = ((int64_t)n_atoms * 32 + 255) / 256;
  PFE_LAUNCH k_filter_matrix<<<(unsigned)blocks, 256, 0, s>>>(n_atoms, rp, ci, H, alpha, shift, out64, out32);
}

void launch_chain_springs(int32_t n_atoms, const int32_t *rp, const int32_t *ci, const double *H, const double *mass,
                          int64_t nbonds, const int32_t *bi, const int32_t *bj, const double *rhat, const double *hbar,
                          double *kbar, double *mbar, cudaStream_t s) {
  if (nbonds > 0) PFE_LAUNCH k_chain_k<<<(unsigned)((nbonds + 255) / 256), 256, 0, s>>>(rp, ci, mass, nbonds, bi, bj, rhat, hbar, kbar);
  if (n_atoms > 0) PFE_LAUNCH k_chain_m<<<(unsigned)((n_atoms + 255) / 256), 256, 0, s>>>(n_atoms, rp, ci, H, mass, hbar, mbar);
}

void launch_outer_accum_seg(const Bsr<double> &pattern, int64_t nnzb, int32_t k, int64_t ld, int32_t nq, int64_t stride,
                            const double *A0, const double *T0, double alpha0, double alpha, double *hbar, cudaStream_t s) {
  if (nq <= 0 || nnzb <= 0 || k <= 0) return;
  const int64_t blocks = (4 * nnzb + 255) / 256;
  PFE_LAUNCH k_outer_accum_seg<<<(unsigned)blocks, 256, 0, s>>>(pattern.n_atoms, nnzb, pattern.rp, pattern.ci, k, ld, nq,
                                                                 stride, A0, T0, alpha0, alpha, hbar);
}

}  // namespace pfe
