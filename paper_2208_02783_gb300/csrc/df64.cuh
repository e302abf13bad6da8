// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2, about 48 significant bits (relative rounding
// ~ 2^-47).  GB300 executes 128 FP32 lanes per SM and clock against two FP64 ones, so
// a stencil that needs FP64-level accuracy runs several times faster on pairs of
// floats than in FP64.  The building blocks are the error-free transformations of
// Knuth (TwoSum: a + b = s + e exactly), Dekker (FastTwoSum, for |a| >= |b|) and the
// FMA form of Dekker's TwoProduct (a b = p + e exactly, e = fma(a, b, -p)); see e.g.
// Muller et al., Handbook of Floating-Point Arithmetic, ch. 4-5, and Hida, Li & Bailey
// (2001) for double-word operations.  Every operation below uses the _rn intrinsics so
// that the compiler neither contracts nor reassociates them.
//
// Storage: a complex df64 value is a float4 (re.hi, re.lo, im.hi, im.lo), 16 bytes like
// a double2.
#pragma once

#include <cuda_runtime.h>

namespace transec {

struct df {
  float hi, lo;
};

__host__ __device__ inline df df_split(double x) {
  const float h = (float)x;
  return df{h, (float)(x - (double)h)};
}
__host__ __device__ inline double df_value(df a) { return (double)a.hi + (double)a.lo; }

__device__ inline df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ inline df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ inline df df_norm(df a) { return fast_two_sum(a.hi, a.lo); }

// a + b with the error bounded relative to the result, |err| <= 3u^2 |a + b| (u = 2^-24;
// Joldes, Muller & Popescu, ACM TOMS 44 (2017), the accurate double-word sum): the
// Krylov updates r - alpha q and r + beta p cancel as the residual falls, and a sum
// whose error scales with |a| + |b| instead costs the solver iterations
__device__ inline df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  const df v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ inline df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ inline df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b, unnormalised: p + e with p = fl(a.hi b.hi) (the caller normalises or
// accumulates); the a.lo b.lo term (~2^-48 relative) is dropped
__device__ inline df df_mul_raw(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df{p, e};
}
__device__ inline df df_mul(df a, df b) {
  const df r = df_mul_raw(a, b);
  return fast_two_sum(r.hi, r.lo);
}
// a * 2^k (exact unless it under- or overflows)
__device__ inline df df_scale(df a, float two_k) { return df{__fmul_rn(a.hi, two_k), __fmul_rn(a.lo, two_k)}; }

// Lazy accumulator: the running hi is kept exact by TwoSum, all rounding errors and
// low parts are gathered in lo, normalised once at the end.
struct dfacc {
  float hi = 0.f, lo = 0.f;
  __device__ inline void add(df t) {
    const df s = two_sum(hi, t.hi);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, t.lo));
  }
  __device__ inline df value() const { return fast_two_sum(hi, lo); }
};

// complex df64
struct dfc {
  df re, im;
};

__device__ inline dfc dfc_load(const float4& v) { return dfc{df{v.x, v.y}, df{v.z, v.w}}; }
__device__ inline float4 dfc_store(const dfc& a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__host__ __device__ inline float4 dfc_from_double2(double2 z) {
  const df r = df_split(z.x), i = df_split(z.y);
  return make_float4(r.hi, r.lo, i.hi, i.lo);
}
__host__ __device__ inline double2 dfc_to_double2(const float4& v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}
__device__ inline dfc dfc_zero() { return dfc{df{0.f, 0.f}, df{0.f, 0.f}}; }

__device__ inline dfc dfc_add(const dfc& a, const dfc& b) { return dfc{df_add(a.re, b.re), df_add(a.im, b.im)}; }

// a * b, complex: (ar br - ai bi) + i (ar bi + ai br), each part one TwoSum of the two
// exact leading products plus the gathered errors
__device__ inline dfc dfc_mul(const dfc& a, const dfc& b) {
  const df p1 = df_mul_raw(a.re, b.re), p2 = df_mul_raw(a.im, b.im);
  const df p3 = df_mul_raw(a.re, b.im), p4 = df_mul_raw(a.im, b.re);
  const df s = two_sum(p1.hi, -p2.hi);
  const df t = two_sum(p3.hi, p4.hi);
  return dfc{fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(p1.lo, p2.lo))),
             fast_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(p3.lo, p4.lo)))};
}

// c + a * b, complex
__device__ inline dfc dfc_fma(const dfc& a, const dfc& b, const dfc& c) { return dfc_add(c, dfc_mul(a, b)); }

// complex bilinear product a * b added to a pair of lazy accumulators
__device__ inline void dfc_dot_add(dfacc& re, dfacc& im, const dfc& a, const dfc& b) {
  const df p1 = df_mul_raw(a.re, b.re), p2 = df_mul_raw(a.im, b.im);
  const df p3 = df_mul_raw(a.re, b.im), p4 = df_mul_raw(a.im, b.re);
  re.add(p1);
  re.add(df_neg(p2));
  im.add(p3);
  im.add(p4);
}

}  // namespace transec
