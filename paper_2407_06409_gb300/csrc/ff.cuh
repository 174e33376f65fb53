// Float-float ("double-single") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  Error-free transformations
// after Dekker (1971) and Knuth (TAOCP vol. 2): two_sum exact by six additions, two_prod
// exact by one product and one FMA.  GB300 runs FP32 about 60x faster than FP64, so a few
// FP32 operations per FP64 operation still relieve the FP64 pipe where 2^-46 relative
// accuracy is enough.
#pragma once

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float hi, float lo) {
  ff r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// nearest float-float of a double (two conversions and one FP64 subtraction)
__device__ __forceinline__ ff ff_from_double(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return ff_make(hi, lo);
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff ff_quick_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff_make(s, e);
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_quick_two_sum(s, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff_make(-a.hi, -a.lo); }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_quick_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

__device__ __forceinline__ ff ff_scale(ff a, float s) {   // a * s for an exact FP32 factor s
  const float p = __fmul_rn(a.hi, s);
  float e = __fmaf_rn(a.hi, s, -p);
  e = __fmaf_rn(a.lo, s, e);
  return ff_quick_two_sum(p, e);
}
