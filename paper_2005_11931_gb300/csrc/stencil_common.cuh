// Device helpers shared by the stencil kernels: 16-byte vector access of a row and the
// arithmetic of one node of B u = cx fx(u) + cy fy(u) (FP32 with fused multiply-adds; FP64 with
// explicitly rounded operations in the order of the definition, no contraction).
#pragma once
#include "tsu_internal.h"

namespace tsu {
namespace dev {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  static constexpr int V = 4;
  using type = float4;
};
template <>
struct Vec<double> {
  static constexpr int V = 2;
  using type = double2;
};

template <typename T>
struct Pack {
  T a[Vec<T>::V];
};

template <typename T>
__device__ __forceinline__ Pack<T> ld_vec(const T* p) {
  Pack<T> r;
  using VT = typename Vec<T>::type;
  VT v = __ldg(reinterpret_cast<const VT*>(p));
  if constexpr (Vec<T>::V == 4) {
    r.a[0] = v.x; r.a[1] = v.y; r.a[2] = v.z; r.a[3] = v.w;
  } else {
    r.a[0] = v.x; r.a[1] = v.y;
  }
  return r;
}

template <typename T>
__device__ __forceinline__ Pack<T> ld_vec_l2(const T* p) {  // data this kernel rewrites and reuses: keep in L2
  Pack<T> r;
  using VT = typename Vec<T>::type;
  VT v = __ldcg(reinterpret_cast<const VT*>(p));
  if constexpr (Vec<T>::V == 4) {
    r.a[0] = v.x; r.a[1] = v.y; r.a[2] = v.z; r.a[3] = v.w;
  } else {
    r.a[0] = v.x; r.a[1] = v.y;
  }
  return r;
}

template <typename T>
__device__ __forceinline__ Pack<T> ld_vec_cg(const T* p) {  // data this kernel also writes (streamed)
  Pack<T> r;
  using VT = typename Vec<T>::type;
  VT v = __ldcs(reinterpret_cast<const VT*>(p));
  if constexpr (Vec<T>::V == 4) {
    r.a[0] = v.x; r.a[1] = v.y; r.a[2] = v.z; r.a[3] = v.w;
  } else {
    r.a[0] = v.x; r.a[1] = v.y;
  }
  return r;
}

template <typename T>
__device__ __forceinline__ void st_vec(T* p, const Pack<T>& r) {
  using VT = typename Vec<T>::type;
  VT v;
  if constexpr (Vec<T>::V == 4) {
    v.x = r.a[0]; v.y = r.a[1]; v.z = r.a[2]; v.w = r.a[3];
  } else {
    v.x = r.a[0]; v.y = r.a[1];
  }
  *reinterpret_cast<VT*>(p) = v;
}

// ---- arithmetic of one node ------------------------------------------------------------------
// FP32: every rounding is explicit (the compiler contracts nothing), so every pass that calls these
// (one step, CTA-blocked, warp-blocked, batched, segment recompute) gives the same bits.
struct ArithF32 {
  float cx, cy;
  __device__ __forceinline__ float b(float hxr, float hxl, float hyu, float hyd, float uc, float ul, float ur,
                                     float uu, float ud) const {
    // fx = hxr (ur - uc) - hxl (uc - ul) written as hxl (ul - uc) + hxr (ur - uc): the form the
    // paired .f32x2 instructions evaluate without a negation
    const float fx = __fmaf_rn(hxl, __fsub_rn(ul, uc), __fmul_rn(hxr, __fsub_rn(ur, uc)));
    const float fy = __fmaf_rn(hyd, __fsub_rn(ud, uc), __fmul_rn(hyu, __fsub_rn(uu, uc)));
    return __fmaf_rn(cx, fx, __fmul_rn(cy, fy));
  }
  __device__ __forceinline__ float lf(float uc, float up, float b) const {
    return __fadd_rn(__fmaf_rn(2.0f, uc, -up), b);
  }
  __device__ __forceinline__ float add(float a, float b) const { return __fadd_rn(a, b); }
};

struct ArithF64 {  // explicitly rounded, definition order, no contraction
  double cx, cy;
  __device__ __forceinline__ double b(double hxr, double hxl, double hyu, double hyd, double uc, double ul,
                                      double ur, double uu, double ud) const {
    double fx = __dsub_rn(__dmul_rn(hxr, __dsub_rn(ur, uc)), __dmul_rn(hxl, __dsub_rn(uc, ul)));
    double fy = __dsub_rn(__dmul_rn(hyu, __dsub_rn(uu, uc)), __dmul_rn(hyd, __dsub_rn(uc, ud)));
    return __dadd_rn(__dmul_rn(cx, fx), __dmul_rn(cy, fy));
  }
  __device__ __forceinline__ double lf(double uc, double up, double b) const {
    return __dadd_rn(__dsub_rn(__dmul_rn(2.0, uc), up), b);
  }
  __device__ __forceinline__ double add(double a, double b) const { return __dadd_rn(a, b); }
};

template <typename T>
struct ArithOf;
template <>
struct ArithOf<float> { using type = ArithF32; };
template <>
struct ArithOf<double> { using type = ArithF64; };

}  // namespace dev
}  // namespace tsu
