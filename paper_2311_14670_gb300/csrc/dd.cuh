// Double-double ("dd") arithmetic: a value is the unevaluated sum hi + lo of two doubles with
// |lo| <= ulp(hi)/2.  Error-free transformations after Dekker (1971) and Knuth (TAOCP vol. 2):
// two_sum (Knuth), fast_two_sum (Dekker, |a| >= |b|), two_prod through a fused multiply-add.
// Division and square root refine a double approximation by one Newton correction in dd.
#pragma once

#include <cuda_runtime.h>

namespace s2gb {

struct dd {
  double hi, lo;
};

__host__ __device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return {s, e};
}

__host__ __device__ __forceinline__ dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__host__ __device__ __forceinline__ dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return {p, e};
}

__host__ __device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  double e = s.lo + (x.lo + y.lo);
  return fast_two_sum(s.hi, e);
}

__host__ __device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }

__host__ __device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

__host__ __device__ __forceinline__ dd dd_mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  double e = p.lo + (x.hi * y.lo + x.lo * y.hi);
  return fast_two_sum(p.hi, e);
}

__host__ __device__ __forceinline__ dd dd_mul_d(dd x, double b) {
  dd p = two_prod(x.hi, b);
  double e = p.lo + x.lo * b;
  return fast_two_sum(p.hi, e);
}

// x / y: q0 = hi/hi, then one correction with the dd remainder.
__host__ __device__ __forceinline__ dd dd_div(dd x, dd y) {
  double q0 = x.hi / y.hi;
  dd r = dd_sub(x, dd_mul_d(y, q0));
  double q1 = r.hi / y.hi;
  dd q = fast_two_sum(q0, q1);
  r = dd_sub(x, dd_mul(y, q));
  double q2 = r.hi / y.hi;
  return dd_add(q, dd{q2, 0.0});
}

// sqrt(x) for x > 0: s0 = sqrt(hi), s = s0 + (x - s0^2) / (2 s0) evaluated in dd.
__host__ __device__ __forceinline__ dd dd_sqrt(dd x) {
  if (x.hi <= 0.0) return {0.0, 0.0};
  double s0 = sqrt(x.hi);
  dd sq = two_prod(s0, s0);
  dd r = dd_sub(x, sq);
  double corr = r.hi / (2.0 * s0);
  return fast_two_sum(s0, corr);
}

__host__ __device__ __forceinline__ dd dd_from_ll(long long v) {
  // exact for |v| < 2^106
  double hi = (double)v;
  double lo = (double)(v - (long long)hi);
  return {hi, lo};
}

}  // namespace s2gb
