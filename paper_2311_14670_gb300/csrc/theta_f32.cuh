// Float32 chain helpers shared by the float32 theta kernels (theta_kernels_f32.cu, FMA-pipe
// contraction; theta_tc.cu, contraction on the tensor cores): starting values from the float64
// routine as a float mantissa and an exponent, dead-chain bookkeeping for float32's narrow range,
// and one step of the unnormalised recursion (plain and difference form, see theta_kernels.cu).
#pragma once

#include "theta_common.cuh"

namespace s2gb {
namespace theta {

constexpr int kLiveThr32 = 90;   // dead while |d| < 2^-90
constexpr int kRescale32 = 20;   // rescale dead chains beyond 2^20 (growth between checks <= 2^14)

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }  // -126..127
__device__ __forceinline__ int expf_of(float x) { return ((__float_as_int(x) >> 23) & 0xff) - 127; }
__device__ __forceinline__ float flipf(float x, unsigned mask) { return __int_as_float(__float_as_int(x) ^ (int)mask); }

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// float64 starting value -> float mantissa x and exponent E (true value x * 2^-E, E = 0 if live)
__device__ __forceinline__ void seed_value_f32(const SeedData& sd, const RingData& rd, float& x, int& E) {
  double xd;
  int Ed;
  seed_value(sd, rd, xd, Ed);
  if (((__double2hiint(xd) & 0x7fffffff) | __double2loint(xd)) == 0) { x = 0.0f; E = 0; return; }
  const int ex = exp_of(xd);
  const int etrue = ex - Ed;
  if (etrue >= -kLiveThr32) {          // then Ed == 0 (float64 dead threshold is lower)
    x = (float)xd;
    E = 0;
  } else {
    x = (float)(xd * pow2i(-ex));      // mantissa in [1, 2)
    E = -etrue;
  }
}

__device__ __forceinline__ void renorm_f32(float& x, float& y, int& E) {
  if (E > 0 && (__float_as_int(x) & 0x7fffffff) != 0) {
    const int ex = expf_of(x);
    if (ex - E >= -kLiveThr32) {       // E <= kRescale32 + 14 + kLiveThr32 < 126
      const float s = pow2f(-E);
      x *= s; y *= s; E = 0;
    } else if (ex > kRescale32) {
      const float s = pow2f(-ex);
      x *= s; y *= s; E -= ex;
    }
  }
}

struct StepCoef32 {
  float A, C, Kn, Ks, Kdn, Kds;
};

template <bool DIFF>
__device__ __forceinline__ void step_f32(float& x, float& y, float v, unsigned north_mask, bool north,
                                         const StepCoef32& c) {
  const float sA = flipf(c.A, north_mask);
  if (!DIFF) {
    const float P = fmaf(sA, v, north ? c.Kn : c.Ks);
    const float xn = fmaf(P, x, -(c.C * y));
    y = x;
    x = xn;
  } else {
    const float Q = fmaf(sA, v, north ? c.Kdn : c.Kds);
    const float sC = flipf(c.C, north_mask ^ 0x80000000u);
    const float en = fmaf(Q, x, sC * y);
    x = fmaf(north ? 1.0f : -1.0f, x, en);
    y = en;
  }
}

}  // namespace theta
}  // namespace s2gb
