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
  if ((rd.pole == 1 && sd.b > 0) || (rd.pole == 2 && sd.a > 0)) { x = 0.0; E = 0; return; }  // cos(pi/2), sin(0)
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

// Coefficients of one step of the normalised recursion (layout of plan.cu's coefn_kernel).
struct StepN {
  double Ap, Knp, Ksp, g, gn, App, Kdnp, Kdsp, en, ig;
};

__device__ __forceinline__ StepN stepn_at(const double* c) {
  return {c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7], c[8], c[9]};
}

// One step of the normalised recursion (2 FP64 instructions plain, 3 in the difference form);
// x, y are (u^j, u^{j-1}) plain (u^j = d^j / gamma_j) or (d^j, ehat^j) in the difference form.
template <bool DIFF>
__device__ __forceinline__ void stepn(double& x, double& y, double v, unsigned nmask, bool north, const StepN& c) {
  if (!DIFF) {
    const double P = fma(flip_sign(c.Ap, nmask), v, north ? c.Knp : c.Ksp);
    const double xn = fma(P, x, -y);
    y = x;
    x = xn;
  } else {
    const unsigned smask = nmask ^ 0x80000000u;          // sign of sigma: + north, - south
    const double Q = fma(flip_sign(c.App, nmask), v, north ? c.Kdnp : c.Kdsp);
    const double en = fma(Q, x, flip_sign(y, smask));     // Q' d + sigma ehat
    x = fma(c.en, en, flip_sign(x, smask));                // sigma d + eta ehat'
    y = en;
  }
}

// Signal slots of a CTA.  Slot b < NB is signal sig0 + b at (m, n); with pairing (PAIR), slot
// NB + b is the same signal at (-m, -n), whose d-functions are d^l_{-m,-n} = (-1)^{m-n} d^l_{m,n}
// (Sec. 3.3 symmetry): the partner column reuses the recursion of (m, n), scaled by that sign.
struct Slot {
  long long sig_off;   // signal offset (sig * nN + ni) or -1 if inactive
  int mi;              // column index m + L - 1 of the slot
  int m;
  double sign;
};

template <int NB, bool PAIR>
__device__ __forceinline__ Slot slot_of(int b, int sig0, int nsig, int nN, int ni, int m, int n, int L) {
  Slot sl;
  const bool partner = PAIR && b >= NB;
  const int sig = sig0 + (partner ? b - NB : b);
  const bool active = sig < nsig && !(partner && m == 0 && n == 0);
  const int nis = partner ? (nN - 1 - ni) : ni;
  sl.m = partner ? -m : m;
  sl.mi = sl.m + L - 1;
  sl.sig_off = active ? (long long)sig * nN + nis : -1;
  sl.sign = (partner && ((m - n) & 1)) ? -1.0 : 1.0;
  return sl;
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
