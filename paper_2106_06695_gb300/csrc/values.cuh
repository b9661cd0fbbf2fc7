// Lattice value storage (fp32 or bf16, converted to fp32 registers) and fp32 register
// vectors of 1 or 4 columns, shared by the MVM and the batched serving kernels.
#pragma once

#include <cuda_bf16.h>
#include <string.h>

namespace sgp {

using bf16 = __nv_bfloat16;

// ---- storage of lattice values: groups of 4 (or 8) values as float4 ------------------
template <class S>
struct Store;

template <>
struct Store<float> {
  static __device__ __forceinline__ float4 ld4(const float* p) {
    return *reinterpret_cast<const float4*>(p);
  }
  static __device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
  }
  static __device__ __forceinline__ void st4(float* p, float4 v) {
    *reinterpret_cast<float4*>(p) = v;
  }
  static __device__ __forceinline__ void ldg8(const float* p, float4& a, float4& b) {
    a = __ldg(reinterpret_cast<const float4*>(p));
    b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  }
  static __device__ __forceinline__ void st8(float* p, float4 a, float4 b) {
    reinterpret_cast<float4*>(p)[0] = a;
    reinterpret_cast<float4*>(p)[1] = b;
  }
  static __device__ __forceinline__ float ld1(const float* p) { return *p; }
  static __device__ __forceinline__ void st1(float* p, float v) { *p = v; }
};

__device__ __forceinline__ float2 unpack2(uint32_t u) {
  __nv_bfloat162 h;
  memcpy(&h, &u, 4);
  return __bfloat1622float2(h);
}
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

template <>
struct Store<bf16> {
  static __device__ __forceinline__ float4 cvt(uint2 u) {
    const float2 a = unpack2(u.x), b = unpack2(u.y);
    return make_float4(a.x, a.y, b.x, b.y);
  }
  static __device__ __forceinline__ float4 ld4(const bf16* p) {
    return cvt(*reinterpret_cast<const uint2*>(p));
  }
  static __device__ __forceinline__ float4 ldg4(const bf16* p) {
    return cvt(__ldg(reinterpret_cast<const uint2*>(p)));
  }
  static __device__ __forceinline__ void st4(bf16* p, float4 v) {
    *reinterpret_cast<uint2*>(p) = make_uint2(pack2(v.x, v.y), pack2(v.z, v.w));
  }
  static __device__ __forceinline__ void ldg8(const bf16* p, float4& a, float4& b) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    a = cvt(make_uint2(u.x, u.y));
    b = cvt(make_uint2(u.z, u.w));
  }
  static __device__ __forceinline__ void st8(bf16* p, float4 a, float4 b) {
    *reinterpret_cast<uint4*>(p) =
        make_uint4(pack2(a.x, a.y), pack2(a.z, a.w), pack2(b.x, b.y), pack2(b.z, b.w));
  }
  static __device__ __forceinline__ float ld1(const bf16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st1(bf16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// x = x1 + x2 + x3 in bf16 (each part the nearest bf16 of what is left; the differences are
// exact in fp32): about 24 significant bits, the three-part operands of the bf16 tensor-core
// products.
__device__ __forceinline__ void split3(float x, bf16& a, bf16& b, bf16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

// ---- fp32 register vectors of VEC = 4 or 1 columns ----------------------------------
template <int VEC>
struct Vec;
template <>
struct Vec<4> {
  using T = float4;
  static __device__ __forceinline__ T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ T ld(const float* p) { return *reinterpret_cast<const float4*>(p); }
  static __device__ __forceinline__ void st(float* p, T v) { *reinterpret_cast<float4*>(p) = v; }
  static __device__ __forceinline__ T ldg(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
  }
  template <class S>
  static __device__ __forceinline__ T lds(const S* p) { return Store<S>::ld4(p); }
  template <class S>
  static __device__ __forceinline__ T ldgs(const S* p) { return Store<S>::ldg4(p); }
  template <class S>
  static __device__ __forceinline__ void sts(S* p, T v) { Store<S>::st4(p, v); }
  static __device__ __forceinline__ T fma(float a, T x, T y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
  }
  static __device__ __forceinline__ T add(T x, T y) {
    return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
  }
  static __device__ __forceinline__ T scale(float a, T x) {
    return make_float4(a * x.x, a * x.y, a * x.z, a * x.w);
  }
};
template <>
struct Vec<1> {
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.f; }
  static __device__ __forceinline__ T ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, T v) { *p = v; }
  static __device__ __forceinline__ T ldg(const float* p) { return __ldg(p); }
  template <class S>
  static __device__ __forceinline__ T lds(const S* p) { return Store<S>::ld1(p); }
  template <class S>
  static __device__ __forceinline__ T ldgs(const S* p) { return Store<S>::ld1(p); }
  template <class S>
  static __device__ __forceinline__ void sts(S* p, T v) { Store<S>::st1(p, v); }
  static __device__ __forceinline__ T fma(float a, T x, T y) { return fmaf(a, x, y); }
  static __device__ __forceinline__ T add(T x, T y) { return x + y; }
  static __device__ __forceinline__ T scale(float a, T x) { return a * x; }
};

}  // namespace sgp
