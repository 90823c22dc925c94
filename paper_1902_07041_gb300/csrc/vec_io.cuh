// Vector loads and stores of CPL adjacent multivector elements (8- or 16-byte lanes), shared by
// the fused step kernels.
#pragma once

namespace pfe {
namespace {

// ---- vector loads/stores of CPL adjacent elements ------------------------------------
__device__ __forceinline__ void ldg_n(const double *p, double (&v)[1]) { v[0] = __ldg(p); }
__device__ __forceinline__ void ldg_n(const double *p, double (&v)[2]) {
  double2 t = __ldg(reinterpret_cast<const double2 *>(p));
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void ldg_n(const float *p, float (&v)[1]) { v[0] = __ldg(p); }
__device__ __forceinline__ void ldg_n(const float *p, float (&v)[2]) {
  float2 t = __ldg(reinterpret_cast<const float2 *>(p));
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void ldg_n(const float *p, float (&v)[4]) {
  float4 t = __ldg(reinterpret_cast<const float4 *>(p));
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ld_n(const double *p, double (&v)[1]) { v[0] = *p; }
__device__ __forceinline__ void ld_n(const double *p, double (&v)[2]) {
  double2 t = *reinterpret_cast<const double2 *>(p);
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void ld_n(const float *p, float (&v)[1]) { v[0] = *p; }
__device__ __forceinline__ void ld_n(const float *p, float (&v)[2]) {
  float2 t = *reinterpret_cast<const float2 *>(p);
  v[0] = t.x;
  v[1] = t.y;
}
__device__ __forceinline__ void ld_n(const float *p, float (&v)[4]) {
  float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void st_n(double *p, const double (&v)[1]) { *p = v[0]; }
__device__ __forceinline__ void st_n(double *p, const double (&v)[2]) {
  *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void st_n(float *p, const float (&v)[1]) { *p = v[0]; }
__device__ __forceinline__ void st_n(float *p, const float (&v)[2]) {
  *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}
__device__ __forceinline__ void st_n(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

}  // namespace
}  // namespace pfe
