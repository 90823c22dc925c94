// A measurement of the machine, not of the method: the FP64 FMA rate the GPU sustains.  Every
// FP64 step of the eigensolver (the filter step, the DMMA Gram and update products) runs on the
// FP64 pipe of GB300, so this rate is the roofline those kernels are reported against.
#include "pfe_internal.h"

namespace pfe {
namespace {

constexpr int kChains = 8;  // independent FMA chains per thread: hides the pipe's latency

__global__ void __launch_bounds__(256) k_fp64_fma_probe(int32_t iters, double *sink) {
  double a[kChains];
  const double b = 1.0 - 1e-12 * (double)(threadIdx.x & 7);
  const double c = 1e-9;
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int32_t t = 0; t < iters; ++t) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.0) *sink = s;  // never true (every chain stays positive); the store keeps the work live
}

}  // namespace
}  // namespace pfe

extern "C" pfe_status pfe_probe_fp64_fma(int32_t iters, int32_t reps, void *stream, double *sink, double *tflops) {
  using namespace pfe;
  if (iters < 1 || reps < 1 || !sink || !tflops) return PFE_E_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PFE_E_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned blocks = (unsigned)sms * 8u;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PFE_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PFE_E_CUDA;
  }
  PFE_LAUNCH k_fp64_fma_probe<<<blocks, 256, 0, s>>>(iters, sink);  // warm-up
  cudaEventRecord(e0, s);
  for (int32_t r = 0; r < reps; ++r) PFE_LAUNCH k_fp64_fma_probe<<<blocks, 256, 0, s>>>(iters, sink);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || ms <= 0.f) return PFE_E_CUDA;
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * 256.0 * (double)reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return PFE_OK;
}
