// Device helpers shared by the float64 and float32 theta kernels (see theta_kernels.cu for the
// recursion, its half-angle / difference forms and the dead-chain bookkeeping).
#pragma once

#include <cuda_runtime.h>

#include "dd.cuh"
#include "s2gb_internal.h"

namespace s2gb {
namespace theta {


constexpr int kLiveThr = 400;   // dead while |d| < 2^-400
constexpr int kRescale = 256;   // rescale dead chains when x exceeds 2^256

__device__ __forceinline__ double pow2i(int e) {          // 2^e, -1022 <= e <= 1023
  return __hiloint2double((1023 + e) << 20, 0);
}
__device__ __forceinline__ int exp_of(double x) {         // unbiased exponent field of x
  return ((__double2hiint(x) >> 20) & 0x7ff) - 1023;
}
__device__ __forceinline__ double flip_sign(double x, unsigned mask) {
  return __hiloint2double(__double2hiint(x) ^ (int)mask, __double2loint(x));
}

// d^{l0}_{m,n}(theta) = sign 2^p sin(theta/2)^a cos(theta/2)^b, evaluated as 2^X with X in
// double-double, returned as x * 2^-E (E = 0 if the value is not tiny).
__device__ __forceinline__ void seed_value(const SeedData& sd, const RingData& rd, double& x, int& E) {
  if ((rd.pole && sd.b > 0)) { x = 0.0; E = 0; return; }      // cos(pi/2) = 0
  dd X = {sd.p_hi, sd.p_lo};
  if (sd.a) {
    dd t = two_prod(rd.ls_hi, (double)sd.a);
    t.lo = fma(rd.ls_lo, (double)sd.a, t.lo);
    X = dd_add(X, t);
  }
  if (sd.b) {
    dd t = two_prod(rd.lc_hi, (double)sd.b);
    t.lo = fma(rd.lc_lo, (double)sd.b, t.lo);
    X = dd_add(X, t);
  }
  double Eh = floor(X.hi);
  double f = (X.hi - Eh) + X.lo;
  if (f < 0.0) { f += 1.0; Eh -= 1.0; }
  if (f >= 1.0) { f -= 1.0; Eh += 1.0; }
  double mant = exp2(f);
  if (sd.sign < 0) mant = -mant;
  int e = (int)Eh;
  if (e >= -kLiveThr) { x = mant * pow2i(e); E = 0; }
  else { x = mant; E = -e; }
}

// Dead-chain bookkeeping (see file comment).  Only touches chains with E > 0.
__device__ __forceinline__ void renorm(double& x, double& y, int& E) {
  if (E > 0 && ((__double2hiint(x) & 0x7fffffff) | __double2loint(x)) != 0) {
    const int ex = exp_of(x);
    if (ex - E >= -kLiveThr) {
      const double s = pow2i(-E);
      x *= s; y *= s; E = 0;
    } else if (ex > kRescale) {
      const double s = pow2i(-ex);
      x *= s; y *= s; E -= ex;
    }
  }
}

struct StepCoef {
  double A, C, Kn, Ks, Kdn, Kds;
};

__device__ __forceinline__ StepCoef load_coef(const double* c) {
  const double2* c2 = reinterpret_cast<const double2*>(c);
  double2 a = __ldg(c2), b = __ldg(c2 + 1), d = __ldg(c2 + 2);
  return {a.x, a.y, b.x, b.y, d.x, d.y};
}

// One recursion step of a chain. north/diff are per-chain constants.
template <bool DIFF>
__device__ __forceinline__ void step(double& x, double& y, double v, unsigned north_mask, bool north,
                                     const StepCoef& c) {
  // sA = -A on north rings, +A on south rings
  const double sA = flip_sign(c.A, north_mask);
  if (!DIFF) {
    const double K = north ? c.Kn : c.Ks;
    const double P = fma(sA, v, K);
    const double xn = fma(P, x, -(c.C * y));
    y = x;
    x = xn;
  } else {
    const double K = north ? c.Kdn : c.Kds;
    const double Q = fma(sA, v, K);
    const double sC = flip_sign(c.C, north_mask ^ 0x80000000u);   // +C north, -C south
    const double en = fma(Q, x, sC * y);
    const double sg = north ? 1.0 : -1.0;                          // sigma
    x = fma(sg, x, en);
    y = en;
  }
}

__device__ __forceinline__ int m_of_rank(int r) {   // 0, -1, 1, -2, 2, ...: longest chains first
  return (r == 0) ? 0 : ((r & 1) ? -((r + 1) >> 1) : (r >> 1));
}

// Ring owned by slot i of thread `tid` in the forward kernel.  The last slot always holds the
// last nt rings (the south polar cap), slot 0 the first nt (the north cap); middle-slot chains that
// would repeat a ring of the last slot are inactive.
template <int KT>
__device__ __forceinline__ int ring_of(int i, int tid, int nt, int L, bool& active) {
  if (KT == 1) { active = tid < L; return tid; }
  if (i == KT - 1) { active = true; return L - nt + tid; }
  const int t = i * nt + tid;
  active = t < L - nt;
  return t;
}

}  // namespace theta
}  // namespace s2gb
