// Node vectors of the cycle are stored 4 values per node (x, y, z, 0) so that a
// node is one aligned 16-byte (FP32) or 32-byte (FP64) access: the gather of
// x_j in a block row is a single vector load.  The pressure part (saddle
// systems) follows the 4n velocity entries as plain scalars.
#pragma once

#include <cuda_runtime.h>

namespace amgp2 {

__device__ __forceinline__ void ld3(const float* p, int j, float& a, float& b, float& c) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p) + j);
  a = v.x; b = v.y; c = v.z;
}

__device__ __forceinline__ void ld3(const double* p, int j, double& a, double& b, double& c) {
  double w;
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
      : "=d"(a), "=d"(b), "=d"(c), "=d"(w)
      : "l"(p + 4 * (size_t)j));
}

// coherent variant for vectors written earlier in the same kernel by other threads
__device__ __forceinline__ void ld3c(const float* p, int j, float& a, float& b, float& c) {
  const float4 v = reinterpret_cast<const float4*>(p)[j];
  a = v.x; b = v.y; c = v.z;
}

__device__ __forceinline__ void ld3c(const double* p, int j, double& a, double& b, double& c) {
  double w;
  asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
               : "=d"(a), "=d"(b), "=d"(c), "=d"(w)
               : "l"(p + 4 * (size_t)j)
               : "memory");
}

__device__ __forceinline__ void st3(float* p, int j, float a, float b, float c) {
  reinterpret_cast<float4*>(p)[j] = make_float4(a, b, c, 0.f);
}

__device__ __forceinline__ void st3(double* p, int j, double a, double b, double c) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p + 4 * (size_t)j), "d"(a),
               "d"(b), "d"(c), "d"(0.0)
               : "memory");
}

// FP32-pair arithmetic of the Krylov operator: (S, s) += a x with a = (a.x, a.y)
// = hi + lo and x = xh + xl.  The product a.x xh is exact as the rounded product
// p plus its error fma(a.x, xh, -p); the cross terms a.x xl + a.y xh join the
// error, a.y xl (about 2^-48 of the product) is dropped; p is added to S with
// TwoSum (Knuth) and the sum's error with the product's error to s.  The _rn
// intrinsics keep the compiler from contracting any of these into an FMA.
__device__ __forceinline__ void pair_fma(float& S, float& s, float2 a, float xh, float xl) {
  const float p = __fmul_rn(a.x, xh);
  float e = fmaf(a.x, xh, -p);
  e = fmaf(a.x, xl, e);
  e = fmaf(a.y, xh, e);
  const float t = __fadd_rn(S, p);
  const float bp = __fsub_rn(t, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  S = t;
  s = __fadd_rn(s, __fadd_rn(err, e));
}

// (S, s) += (T, t) for the reduction across the lanes of a row
__device__ __forceinline__ void pair_add(float& S, float& s, float T, float t) {
  const float u = __fadd_rn(S, T);
  const float bp = __fsub_rn(u, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(u, bp)), __fsub_rn(T, bp));
  S = u;
  s = __fadd_rn(s, __fadd_rn(err, t));
}

}  // namespace amgp2
