// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two float32 numbers with |lo| <= ulp(hi)/2, giving about 48 significand
// bits on the FP32 pipes.  The building blocks are the classical error-free
// transformations: Knuth's TwoSum, Dekker's Fast2Sum, and the exact product
// a*b = p + fma(a, b, -p).  All float operations use the _rn intrinsics, which
// the compiler never contracts into fused multiply-adds, so every rounding is
// the one the algorithm assumes.
//
// Why: the per-oscillator torque of Eq. (gov) needs more than FP32 (float32
// rounding along a periodic orbit biases the precession frequency and breaks
// a 1e-4 parity bar within 200 input samples), while FP64 runs at 1/64 of
// the FP32 rate on this part and put ~2 us per stage on the critical path.
#pragma once

#include <cuda_runtime.h>

namespace sto {

struct df {
  float hi, lo;
};

// Host: split a double into hi + lo.
inline df df_split_host(double x) {
  const float hi = static_cast<float>(x);
  return {hi, static_cast<float>(x - static_cast<double>(hi))};
}

__device__ __forceinline__ df df_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - static_cast<double>(hi))};
}

__device__ __forceinline__ double df_to_double(df a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}

__device__ __forceinline__ df df_from(float x) { return {x, 0.f}; }

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

// p + e = a * b exactly.
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// Sum of two df values.  The error is below about 2^-46 (|a| + |b|): an
// absolute bound on the scale of the operands, which is what the torque
// needs (its terms are O(1) x O(|b|)); exact cancellation is not required.
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// Sum of a df and a float.
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// a * b without the final renormalisation: hi + lo carries the product to
// the same accuracy as df_mul, with |lo| up to a few ulp(hi).  Only an
// operand of df_add / df_mul (which renormalise), never a stored value.
__device__ __forceinline__ df df_mul_raw(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return p;
}

// c + a * b.
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(c, df_mul_raw(a, b)); }

// Exact scaling by a power of two.
__device__ __forceinline__ df df_scale2(df a, float pow2) {
  return {__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)};
}

// a*b - c*d (one component of a cross product).
__device__ __forceinline__ df df_cross1(df a, df b, df c, df d) {
  return df_sub(df_mul_raw(a, b), df_mul_raw(c, d));
}

// Terms of the spin-torque field that depend on the polarizer p: m . p and
// p x m.  The paper's p = (1, 0, cos 90 deg) has p_y = 0 exactly; its terms
// are then left out (a uniform branch on a launch constant).
__device__ __forceinline__ void df_p_terms(df px, df py, df pz, const df m[3], df* s, df c[3]) {
  if (py.hi == 0.f && py.lo == 0.f) {
    *s = df_add(df_mul_raw(m[0], px), df_mul_raw(m[2], pz));
    c[0] = df_neg(df_mul(pz, m[1]));
    c[1] = df_cross1(pz, m[0], px, m[2]);
    c[2] = df_mul(px, m[1]);
  } else {
    *s = df_add(df_add(df_mul_raw(m[0], px), df_mul_raw(m[1], py)), df_mul_raw(m[2], pz));
    c[0] = df_cross1(py, m[2], pz, m[1]);
    c[1] = df_cross1(pz, m[0], px, m[2]);
    c[2] = df_cross1(px, m[1], py, m[0]);
  }
}

// 1 / b: float reciprocal refined by one Newton step in df.
__device__ __forceinline__ df df_rcp(df b) {
  const float q = __frcp_rn(b.hi);
  // r = 1 - q*b, computed in df
  const df qb = df_mul_f(b, q);
  const df r = df_add_f(df_neg(qb), 1.0f);
  // q + q*r
  const df corr = two_prod(q, r.hi);
  return fast_two_sum(q, __fadd_rn(corr.hi, __fmaf_rn(q, r.lo, corr.lo)));
}

}  // namespace sto
