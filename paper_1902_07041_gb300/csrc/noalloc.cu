// pfe_filter_apply_noalloc: the Chebyshev filter of pfe_filter_apply with every work buffer
// taken from one file-scope device array instead of cudaMalloc.
//
// Who needs it: applications that cannot let a library allocate device memory while they run --
// for example when another allocator (a framework's caching allocator, or a pool sized at start-up)
// already owns the device memory, or in loops that cannot afford the implicit device
// synchronisation that cudaMalloc and cudaFree may cause.
//
// The scratch array holds PFE_NOALLOC_MAX_DOUBLES doubles (32 MiB).  It is a property of the loaded
// library: every GPU that loads it keeps the array until the process exits, and every call shares
// it, keeping the contents of the last call.  Calls that overlap on the GPU (other streams, other
// host threads) therefore race on it; the caller serialises them.
#include <cmath>

#include "pfe_internal.h"

#define PFE_NOALLOC_MAX_DOUBLES (4 * 1024 * 1024)

namespace {

__device__ __align__(256) double g_noalloc_scratch[PFE_NOALLOC_MAX_DOUBLES];

// Device address of the scratch array, looked up once per device (with that device current).
constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" pfe_status pfe_filter_apply_noalloc(pfe_ctx *ctx, int32_t m, const double *coeffs, int32_t k,
                                               const double *X, int64_t ldx, double *Y, int64_t ldy, void *stream) {
  using namespace pfe;
  if (!ctx) return PFE_E_ARG;
  if (!coeffs || m < 0 || k < 0 || (k > 0 && (!X || !Y)) || ldx < ctx->n || ldy < ctx->n)
    return pfe_fail(ctx, PFE_E_ARG, "filter_apply_noalloc: bad arguments");
  if (k == 0) return PFE_OK;
  for (int32_t j = 0; j <= m; ++j)
    if (!std::isfinite(coeffs[j])) return pfe_fail(ctx, PFE_E_ARG, "filter_apply_noalloc: non-finite coefficient");
  const int64_t n = ctx->n, ld = (k + 3) / 4 * 4;
  const int64_t need = 4 * n * ld;  // row-major copies of X and Y, two recurrence buffers
  if (need > PFE_NOALLOC_MAX_DOUBLES)
    return pfe_fail(ctx, PFE_E_CAPACITY,
                    "filter_apply_noalloc: 4 * n * round_up(k, 4) = " + std::to_string(need) +
                        " doubles exceeds the fixed scratch of " + std::to_string(PFE_NOALLOC_MAX_DOUBLES));
  if (!ctx->has_lmax || !ctx->hs_valid || ctx->hs_c != ctx->tc || ctx->hs_d != ctx->td)
    return pfe_fail(ctx, PFE_E_STATE,
                    "filter_apply_noalloc: the context has no FP64 filter operator yet (one pfe_filter_apply, "
                    "pfe_estimate or pfe_solve call builds it)");
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return pfe_fail(ctx, PFE_E_ARG, "device ordinal out of range");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, "cudaSetDevice failed");
  // first call on this device: resolve the array's device address (no allocation)
  if (!g_scratch_ptr[ctx->device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return pfe_fail(ctx, PFE_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[ctx->device] = static_cast<double *>(p);
  }
  double *base = g_scratch_ptr[ctx->device];
  double *Xr = base, *Yr = base + n * ld, *b0 = base + 2 * n * ld, *b1 = base + 3 * n * ld;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
  // the filter operator was built on the context's stream: wait for it (a host wait, no allocation)
  if (s != ctx->stream) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  }
  // The array keeps the previous call's contents.  Columns are independent, so only the padding
  // columns k .. ld-1 of the four blocks (read by the vector lanes, never copied out) are cleared.
  if (ld > k) {
    for (double *p : {Xr, Yr, b0, b1}) {
      cudaError_t e = cudaMemset2DAsync(p + k, (size_t)ld * sizeof(double), 0, (size_t)(ld - k) * sizeof(double),
                                        (size_t)n, s);
      if (e != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, std::string("cudaMemset2DAsync: ") + cudaGetErrorString(e));
    }
  }
  launch_colmajor_to_rowmajor<double>(n, k, X, ldx, Xr, ld, s);
  // the filter driver of pfe_filter_apply (rank-1 operator when built, STEP / STEP_ACC launches),
  // without its shape autotuner, which would synchronise the stream
  PFE_TRY(solver_filter64_rows(ctx, coeffs, m, k, ld, Xr, Yr, b0, b1, s, false));
  launch_rowmajor_to_colmajor<double>(n, k, Yr, ld, Y, ldy, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfe_fail(ctx, PFE_E_CUDA, std::string("filter_apply_noalloc: ") + cudaGetErrorString(e));
  return PFE_OK;
}
