// Two-lane FP32 arithmetic for kernels that update two nodes per thread.
// Every operation maps to one packed instruction of the sm_100 family
// (fma.rn.f32x2, add.rn.f32x2, mul.rn.f32x2), each lane rounded exactly as
// the scalar operation would be.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstring>

#include "node.cuh"

namespace lbm {

struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ F2(float2 a) : v(a) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ static F2 splat(float a) { return F2(a, a); }
  __device__ __forceinline__ float x() const { return v.x; }
  __device__ __forceinline__ float y() const { return v.y; }
};

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  return F2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y)));
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }

// c * v for a compile-time lattice coefficient c.
template <int C> __device__ __forceinline__ F2 cmul2(F2 v) {
  if constexpr (C == 0) return F2::splat(0.f);
  else if constexpr (C == 1) return v;
  else if constexpr (C == -1) return -v;
  else return v * F2::splat((float)C);
}
template <int CX, int CY> __device__ __forceinline__ F2 cdot2(F2 ux, F2 uy) {
  if constexpr (CX == 0) return cmul2<CY>(uy);
  else if constexpr (CY == 0) return cmul2<CX>(ux);
  else return cmul2<CX>(ux) + cmul2<CY>(uy);
}

// Two adjacent stored values as an F2 (load, load1) and back (store_rn,
// store_sr): FP32 storage moves f; FP16S / BF16S move the scaled deviation h
// (see the codecs in node.cuh), converted exactly to FP32 and rounded back to
// 16 bits, to nearest-even or stochastically.
template <typename S> struct Pair;
template <> struct Pair<__half> {
  using Raw = __half2;
  __device__ __forceinline__ static __half lane(Raw r, int e) { return e ? __high2half(r) : __low2half(r); }
  __device__ __forceinline__ static F2 load(Raw r) { return F2(__half22float2(r)); }
  __device__ __forceinline__ static F2 load1(__half a, __half b) {
    return F2(__half2float(a), __half2float(b));
  }
  __device__ __forceinline__ static Raw store_rn(F2 h) { return __floats2half2_rn(h.x(), h.y()); }
  // Stochastic rounding of both lanes from one random word r (first node in
  // the low half).
  __device__ __forceinline__ static Raw store_sr(F2 h, uint32_t r) {
    const uint32_t u = cvt_rs_f16x2(h.y(), h.x(), r);
    Raw out;
    static_assert(sizeof(out) == sizeof(u), "half2 is 32 bits");
    memcpy(&out, &u, sizeof u);
    return out;
  }
};
template <> struct Pair<__nv_bfloat16> {
  using Raw = __nv_bfloat162;
  __device__ __forceinline__ static __nv_bfloat16 lane(Raw r, int e) {
    return e ? __high2bfloat16(r) : __low2bfloat16(r);
  }
  __device__ __forceinline__ static F2 load(Raw r) { return F2(__bfloat1622float2(r)); }
  __device__ __forceinline__ static F2 load1(__nv_bfloat16 a, __nv_bfloat16 b) {
    return F2(__bfloat162float(a), __bfloat162float(b));
  }
  __device__ __forceinline__ static Raw store_rn(F2 h) { return __floats2bfloat162_rn(h.x(), h.y()); }
  __device__ __forceinline__ static Raw store_sr(F2 h, uint32_t r) {
    const uint32_t u = cvt_rs_bf16x2(h.y(), h.x(), r);
    Raw out;
    static_assert(sizeof(out) == sizeof(u), "bfloat162 is 32 bits");
    memcpy(&out, &u, sizeof u);
    return out;
  }
};
template <> struct Pair<float> {
  using Raw = float2;
  __device__ __forceinline__ static float lane(Raw r, int e) { return e ? r.y : r.x; }
  __device__ __forceinline__ static F2 load(Raw r) { return F2(r); }
  __device__ __forceinline__ static F2 load1(float a, float b) { return F2(a, b); }
  __device__ __forceinline__ static Raw store_rn(F2 f) { return f.v; }
  __device__ __forceinline__ static Raw store_sr(F2 f, uint32_t) { return f.v; }
};

}  // namespace lbm
