// Float-float ("double-float") arithmetic on pairs of float32, and exact conversions
// between float64 bit patterns and float32 pairs done with integer instructions.
//
// GB300 runs float64 arithmetic and float32<->float64 conversions at about 1/64 of
// the float32 rate, so the refinement path keeps float64 off its hot loop: a value is
// carried as hi + lo (two float32) and combined with error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2):  s = a + b exactly as s + e
//   FastTwoSum (Dekker 1971), valid when |a| >= |b|
//   TwoProd with fused multiply-add:      p = a * b exactly as p + e
// All steps use the _rn intrinsics so that the compiler cannot contract or reorder
// them.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace shen {
namespace df {

struct F2 {      // value = hi + lo
    float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// x + y, both float-float; result renormalised.
__device__ __forceinline__ F2 add(F2 x, F2 y) {
    F2 s = two_sum(x.hi, y.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, lo);
}

// x + b with b a float32.
__device__ __forceinline__ F2 add(F2 x, float b) {
    F2 s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

// x * y (float-float times float-float), unnormalised result (hi, lo).
__device__ __forceinline__ F2 mul(F2 x, F2 y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return {p, e};
}

// x * b (float-float times float32).
__device__ __forceinline__ F2 mul(F2 x, float b) {
    const float p = __fmul_rn(x.hi, b);
    float e = __fmaf_rn(x.hi, b, -p);
    e = __fmaf_rn(x.lo, b, e);
    return {p, e};
}

// float64 -> float-float with integer instructions only (no float64 pipe).
// hi = the float64 truncated to a 24-bit significand, lo = the next 23 bits, so
// |d - (hi + lo)| <= 2^-47 |d|.  Magnitudes below 2^-126 give 0 (absolute error
// < 1.2e-38); for |d| < 2^-80 the lo part is dropped (absolute error < 2^-103).
// |d| >= 2^128 is outside float range and gives +-inf.
__device__ __forceinline__ F2 from_f64(double d) {
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t hi32 = (uint32_t)(b >> 32), lo32 = (uint32_t)b;
    const uint32_t sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7FFu);
    uint32_t hb = __funnelshift_l(lo32, hi32 - (896u << 20), 3);
    hb = (hb & 0x7FFFFFFFu) | sign;
    const uint32_t m23 = (lo32 >> 6) & 0x7FFFFFu;
    const float lf = __fsub_rn(__uint_as_float(0x4B000000u | m23), 8388608.0f);
    const int pe = e - 942;                                  // float exponent field of 2^(E-46)
    const float scale = __uint_as_float((uint32_t)max(pe, 0) << 23);
    const float lo = __uint_as_float(__float_as_uint(__fmul_rn(lf, scale)) | sign);
    F2 r;
    r.hi = e >= 897 ? (e <= 1150 ? __uint_as_float(hb) : __uint_as_float(sign | 0x7F800000u))
                    : __uint_as_float(sign);
    r.lo = (e >= 897 && e <= 1150) ? lo : 0.0f;
    return r;
}

// float64 -> float32 by truncation of the significand (the hi part of from_f64),
// integer instructions only.  Same range rules as from_f64.
__device__ __forceinline__ float hi_f64(double d) {
    const uint64_t b = (uint64_t)__double_as_longlong(d);
    const uint32_t hi32 = (uint32_t)(b >> 32), lo32 = (uint32_t)b;
    const uint32_t sign = hi32 & 0x80000000u;
    const uint32_t e = (hi32 >> 20) & 0x7FFu;
    const uint32_t hb = (__funnelshift_l(lo32, hi32 - (896u << 20), 3) & 0x7FFFFFFFu) | sign;
    return __uint_as_float(e - 897u <= 253u ? hb : (e > 1150u ? (sign | 0x7F800000u) : sign));
}

// float32 -> float64 bit pattern with integer instructions (exact for normal floats;
// zero and subnormals give a signed zero).
__device__ __forceinline__ double f32_to_f64_bits(float x) {
    const uint32_t xb = __float_as_uint(x);
    const uint32_t mag = xb & 0x7FFFFFFFu;
    const uint32_t sign = xb & 0x80000000u;
    const bool normal = mag >= 0x00800000u;
    const uint32_t hi32 = normal ? (((mag >> 3) + (896u << 20)) | sign) : sign;
    const uint32_t lo32 = normal ? (mag << 29) : 0u;
    return __longlong_as_double((long long)(((uint64_t)hi32 << 32) | lo32));
}

// float-float -> float64: both parts widened by integer instructions, then one
// float64 addition (the only float64-pipe instruction of the conversion).
__device__ __forceinline__ double to_f64(F2 x) {
    return __dadd_rn(f32_to_f64_bits(x.hi), f32_to_f64_bits(x.lo));
}

}  // namespace df
}  // namespace shen
