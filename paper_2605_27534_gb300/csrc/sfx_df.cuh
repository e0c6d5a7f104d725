// Double-float arithmetic for SFX_F32 contexts: a value is a float2
// (x = hi, y = lo) with value hi + lo and |lo| <= ulp(hi)/2, about 48
// significant bits.  Only FP32 instructions are used: GB300 executes FP64
// at 1/64 of its FP32 rate, so the hot loops never touch the FP64 pipe.
// Error-free transformations after Knuth (two-sum) and Dekker
// (fast two-sum).
#pragma once

#include <cuda_runtime.h>

namespace sfx {

__device__ __forceinline__ float2 ef_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ float2 ef_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return make_float2(s, e);
}

// (hi, lo) + b, renormalised
__device__ __forceinline__ float2 df_add(float2 a, float b) {
  float2 s = ef_two_sum(a.x, b);
  return ef_fast_two_sum(s.x, __fadd_rn(s.y, a.y));
}

// (hi, lo) + (hi, lo), renormalised
__device__ __forceinline__ float2 df_add2(float2 a, float2 b) {
  float2 s = ef_two_sum(a.x, b.x);
  return ef_fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}

// a - b rounded to float: exact leading part when a and b are close
__device__ __forceinline__ float df_diff(float2 a, float2 b) {
  return __fadd_rn(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
}

__device__ __forceinline__ float df_val(float2 a) { return __fadd_rn(a.x, a.y); }

}  // namespace sfx

namespace sfx {

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// a - b as a pair
__device__ __forceinline__ float2 df_sub2(float2 a, float2 b) { return df_add2(a, df_neg(b)); }

// pair times float (Dekker product through fma)
__device__ __forceinline__ float2 df_mul_f(float2 a, float b) {
  float p = __fmul_rn(a.x, b);
  float e = fmaf(a.x, b, -p);
  e = fmaf(a.y, b, e);
  return ef_fast_two_sum(p, e);
}

// pair times pair
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return ef_fast_two_sum(p, e);
}

// pair divided by float
__device__ __forceinline__ float2 df_div_f(float2 a, float b) {
  float q1 = __fdiv_rn(a.x, b);
  float p = __fmul_rn(q1, b);
  float pe = fmaf(q1, b, -p);
  float r = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), pe), a.y);
  return ef_fast_two_sum(q1, __fdiv_rn(r, b));
}

// Folded phase field of SFX_F32 contexts: s = phi for phi <= 1/2 and
// s = phi - 1 (sign bit set) for phi > 1/2, so that both phi and 1 - phi
// keep full relative precision in one float.
struct PhiPair {
  float p, q;   // phi, 1 - phi
};

__device__ __forceinline__ PhiPair unfold(float s) {
  return signbit(s) ? PhiPair{__fadd_rn(1.0f, s), -s} : PhiPair{s, __fsub_rn(1.0f, s)};
}

}  // namespace sfx
