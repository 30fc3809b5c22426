// flb_lane.cuh -- lane-generic FP32 arithmetic for the per-site kernels.
//
// F1 holds one site's value; F2 holds two sites' values in one 64-bit register
// pair and computes with Blackwell's packed FP32 instructions (add/mul/fma on
// f32x2: one issue slot for two lanes).  Every operation of both types is an
// explicitly rounded IEEE operation, so a kernel written once over V gives the
// same bits lane by lane whether it runs one site per thread (F1) or two (F2).
//
// One exception, measured with nvcc 13.0 for sm_103a: a packed product whose
// one factor is a scalar broadcast to both lanes (x * s), followed by a packed
// add of that product, may be fused by the code generator into one packed FMA
// (with the intrinsics and with .rn inline PTX alike); scalar .rn operations
// never are, and neither is a product of two lane-wise values.  A product by a
// scalar that must stay rounded before it is added (a non-exact s) is therefore
// formed by vmul_sep, one scalar multiply per lane.  Products by -1 or a power
// of two are exact and need no care.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace flb {

struct F1 {
    float v;
    static constexpr int L = 1;
    __device__ __forceinline__ static F1 bc(float s) { return F1{s}; }
    __device__ __forceinline__ float lane(int) const { return v; }
};

struct F2 {
    float2 v;
    static constexpr int L = 2;
    __device__ __forceinline__ static F2 bc(float s) { return F2{make_float2(s, s)}; }
    __device__ __forceinline__ float lane(int l) const { return l ? v.y : v.x; }
};

__device__ __forceinline__ F1 mk1(const float *s) { return F1{s[0]}; }
__device__ __forceinline__ F2 mk2(const float *s) { return F2{make_float2(s[0], s[1])}; }
template <class V>
__device__ __forceinline__ V vmake(const float *s);
template <>
__device__ __forceinline__ F1 vmake<F1>(const float *s) { return mk1(s); }
template <>
__device__ __forceinline__ F2 vmake<F2>(const float *s) { return mk2(s); }

__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return F1{__fadd_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 operator+(F1 a, float s) { return F1{__fadd_rn(a.v, s)}; }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return F1{__fsub_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return F1{__fmul_rn(a.v, b.v)}; }
__device__ __forceinline__ F1 operator*(F1 a, float s) { return F1{__fmul_rn(a.v, s)}; }
__device__ __forceinline__ F1 operator*(float s, F1 a) { return F1{__fmul_rn(s, a.v)}; }
__device__ __forceinline__ F1 vfma(F1 a, F1 b, F1 c) { return F1{__fmaf_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F1 vfma(F1 a, float b, F1 c) { return F1{__fmaf_rn(a.v, b, c.v)}; }
__device__ __forceinline__ F1 vfma(float a, F1 b, F1 c) { return F1{__fmaf_rn(a, b.v, c.v)}; }

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator+(F2 a, float s) { return F2{__fadd2_rn(a.v, make_float2(s, s))}; }
// a - b = round(b * (-1) + a): the product is exact, so this is the rounded difference
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2{__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, float s) { return F2{__fmul2_rn(a.v, make_float2(s, s))}; }
__device__ __forceinline__ F2 operator*(float s, F2 a) { return F2{__fmul2_rn(make_float2(s, s), a.v)}; }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return F2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 vfma(F2 a, float b, F2 c) { return F2{__ffma2_rn(a.v, make_float2(b, b), c.v)}; }
__device__ __forceinline__ F2 vfma(float a, F2 b, F2 c) { return F2{__ffma2_rn(make_float2(a, a), b.v, c.v)}; }

// x * s rounded in every lane, never fused with a later add
__device__ __forceinline__ F1 vmul_sep(F1 a, float s) { return F1{__fmul_rn(a.v, s)}; }
__device__ __forceinline__ F2 vmul_sep(F2 a, float s)
{
    return F2{make_float2(__fmul_rn(a.v.x, s), __fmul_rn(a.v.y, s))};
}

}  // namespace flb
