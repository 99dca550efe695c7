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
//
// Forward passes: the face fluxes F = h (u_right - u_left) are rounded once each and B u is their
// difference, fx = F(i+1/2) - F(i-1/2), so that neighbouring nodes share each face's flux (the
// warp-blocked pass computes every flux once and takes the one left of a lane from its
// neighbour), then B u = fma(cx, fx, cy fy).
struct ArithF32 {
  float cx, cy;
  __device__ __forceinline__ float b(float hxr, float hxl, float hyu, float hyd, float uc, float ul, float ur,
                                     float uu, float ud) const {
    const float fx = __fsub_rn(__fmul_rn(hxr, __fsub_rn(ur, uc)), __fmul_rn(hxl, __fsub_rn(uc, ul)));
    const float fy = __fsub_rn(__fmul_rn(hyu, __fsub_rn(uu, uc)), __fmul_rn(hyd, __fsub_rn(uc, ud)));
    return __fmaf_rn(cx, fx, __fmul_rn(cy, fy));
  }
  __device__ __forceinline__ float lf(float uc, float up, float b) const {
    return __fadd_rn(__fmaf_rn(2.0f, uc, -up), b);
  }
  __device__ __forceinline__ float add(float a, float b) const { return __fadd_rn(a, b); }
};

// The one-step adjoint pass: B lambda with one fused multiply-add per direction,
// fx = fma(hxl, ul - uc, hxr (ur - uc)), B = fma(cx, fx, cy fy).  (The four-step adjoint pass
// evaluates B lambda in flux form, like the forward passes; the two round differently, within
// the FP32 adjoint's tolerance.)
struct ArithF32Fma {
  float cx, cy;
  __device__ __forceinline__ float b(float hxr, float hxl, float hyu, float hyd, float uc, float ul, float ur,
                                     float uu, float ud) const {
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

// Four consecutive columns as two packed pairs (c0, c1), (c2, c3) for the paired FP32
// instructions of the sm_100 family (mul/fma .f32x2): two columns per instruction, each element
// rounded exactly as the scalar ArithF32 helper rounds it.
typedef unsigned long long f2x;
struct P4 {
  f2x p[2];
};
__device__ __forceinline__ f2x pk(float lo, float hi) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk(f2x a) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
  return r;
}
// Additions and subtractions run as two scalar instructions: on the warp-blocked pass that
// measured faster than the paired forms (8192^2: 793 against 767 GLUPS; paired multiplies and
// fused multiply-adds do pay: 770 with scalar multiplies, 692 with everything scalar).
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  const float2 x = upk(a), y = upk(b);
  return pk(__fadd_rn(x.x, y.x), __fadd_rn(x.y, y.y));
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  const float2 x = upk(a), y = upk(b);
  return pk(__fsub_rn(x.x, y.x), __fsub_rn(x.y, y.y));
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ P4 lds_p4(const float* s) {
  const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(s);
  return P4{{v.x, v.y}};
}
__device__ __forceinline__ void stg_p4(float* g, const P4& v) {
  *reinterpret_cast<ulonglong2*>(g) = make_ulonglong2(v.p[0], v.p[1]);
}
constexpr P4 kZeroP4{{0ull, 0ull}};  // +0.0f in every column

template <typename T>
struct ArithOf;
template <>
struct ArithOf<float> { using type = ArithF32; };
template <>
struct ArithOf<double> { using type = ArithF64; };
template <typename T>
struct AdjArithOf;
template <>
struct AdjArithOf<float> { using type = ArithF32Fma; };
template <>
struct AdjArithOf<double> { using type = ArithF64; };

}  // namespace dev
}  // namespace tsu
