// A measurement of the machine, not of the method: the FP64 rate the GPU sustains.  Every FP64
// step of the eigensolver (the filter step, the DMMA Gram and update products) runs on the FP64
// pipe of GB300, so this rate is the roofline those kernels are reported against.
#include "pfe_internal.h"

namespace pfe {
namespace {

// CHAINS independent chains per thread hide the pipe's latency.  MIX = 0: every instruction is an
// FMA; MIX = 1: FMA chains and multiply chains alternate (the instruction mix of the filter step,
// whose dot products start with a multiply).  Rates count 2 flops per FP64 instruction, the
// convention of the filter's own flop count (each FMA, and each multiply that starts a dot product).
// MIX = 2: FMAs whose multiplier and addend differ per chain (no operand shared between chains).
template <int CHAINS, int MIX>
__global__ void __launch_bounds__(256) k_fp64_probe(int32_t iters, double *sink) {
  double a[CHAINS], b[CHAINS], c[CHAINS];
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) {
    a[i] = (double)(threadIdx.x + i) * 1e-3 + 0.5;
    b[i] = 1.0 - 1e-12 * (double)((threadIdx.x + (MIX == 2 ? i : 0)) & 7);
    c[i] = 1e-9 * (MIX == 2 ? (double)(i + 1) : 1.0);
  }
  for (int32_t t = 0; t < iters; ++t) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (MIX == 1 && (i & 1)) ? a[i] * b[i] : fma(a[i], b[i], c[i]);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) s += a[i];
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
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PFE_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PFE_E_CUDA;
  }
  double best = 0.0;
  cudaError_t err = cudaSuccess;
  // shapes: {chains, mix, CTAs per SM}
  const int shapes[][3] = {{8, 0, 8}, {16, 0, 8}, {8, 0, 4}, {16, 0, 4}, {8, 1, 8}, {16, 1, 8}, {8, 2, 8}, {8, 2, 4}};
  for (const auto &sh : shapes) {
    const unsigned blocks = (unsigned)sms * (unsigned)sh[2];
    auto launch = [&]() {
      if (sh[1] == 2) PFE_LAUNCH k_fp64_probe<8, 2><<<blocks, 256, 0, s>>>(iters, sink);
      else if (sh[0] == 8 && sh[1] == 0) PFE_LAUNCH k_fp64_probe<8, 0><<<blocks, 256, 0, s>>>(iters, sink);
      else if (sh[0] == 16 && sh[1] == 0) PFE_LAUNCH k_fp64_probe<16, 0><<<blocks, 256, 0, s>>>(iters, sink);
      else if (sh[0] == 8) PFE_LAUNCH k_fp64_probe<8, 1><<<blocks, 256, 0, s>>>(iters, sink);
      else PFE_LAUNCH k_fp64_probe<16, 1><<<blocks, 256, 0, s>>>(iters, sink);
    };
    launch();  // warm-up
    cudaEventRecord(e0, s);
    for (int32_t r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess || ms <= 0.f) break;
    const double fpt = 2.0 * sh[0] * (double)iters;  // 2 per FP64 instruction
    const double rate = fpt * (double)blocks * 256.0 * (double)reps / (ms * 1e-3) / 1e12;
    best = rate > best ? rate : best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || best <= 0.0) return PFE_E_CUDA;
  *tflops = best;
  return PFE_OK;
}
