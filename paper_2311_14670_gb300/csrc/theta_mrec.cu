// Theta stages with the paper's own recursion over the order m (Sec. 3.3, Eq. "wigner-d-recursion"):
//     d^l_{m-1,n}(b) = lambda_m a_{m-1} d^l_{m,n}(b) - (a_{m-1}/a_m) d^l_{m+1,n}(b),
//     lambda_m = (n - m cos b) / sin b,    a_m = 2 / sqrt((l-m)(l+m+1)),
// started at m = l from Eq. "initial_values" (d^l_{l+1,n} = 0) and run downward in m for every
// (l, theta) pair independently -- the plan flag S2GB_PLAN_MRECURSION selects these kernels in
// place of the degree-recursion kernels of theta_kernels.cu.
//
// Stability.  Downward from m = l a chain starts in the region where the wanted solution grows
// (towards smaller m) and enters the oscillatory one; past its lower turning point it would decay
// and rounding errors would grow.  Each (l, theta) is therefore covered by two chains (the same
// reading as the oracle's): chain A at b for m >= m* = rint(n cos b), the middle of the oscillatory
// region, and chain B at pi - b for the rest through d^l_{m,n}(b) = (-1)^{l+n} d^l_{-m,n}(pi - b).
// For n = 0 chain B is not needed: d^l_{-m,0} = (-1)^m d^l_{m,0} (Sec. 3.3 symmetries), and the
// orders -m come from chain A with that sign.
//
// Arithmetic.  lambda_m is evaluated from the ring's half-angle variable v (2 sin^2(b/2) north,
// 2 cos^2(b/2) south): n - m cos b = (n - m) + m v (north) or (n + m) - m v (south), times 1/sin b
// -- cos b itself cannot resolve b near the poles.  a_{m-1} and a_{m-1}/a_m are per (l, m) and come
// from a plan table built in double-double.  A step costs 3 FP64 instructions (lambda a, the
// product with d_{m+1}, one FMA).  Starting values (Eq. initial_values, in log space) and the dead
// chain bookkeeping (values x 2^-E below 2^-400 contribute nothing; exact power-of-two rescaling)
// are those of the degree-recursion kernels (theta_common.cuh); the paper's every-step running
// normalisation becomes this exact power-of-two exponent, checked every 8 steps.
//
// Thread mapping.  The recursion variable m is also the output index of both contractions, so the
// sums run across chains:
//   inverse  ftilde_m(t) = sum_l h_{l,m} d^l_m(t): a lane owns one ring and 16 chains of 16
//            consecutive degrees (the sum over those degrees is in-thread), the 2 warps of a CTA
//            own 32 degrees of the same 32 rings and are summed through shared memory in a fixed
//            order; each CTA writes its 32-degree partial, and a fixed-order sum over the partials
//            gives ftilde (deterministic).
//   forward  flm_{l,m} = sum_t g_m(t) d^l_m(t): a lane owns one degree and 16 chains of 16 rings
//            (the sum over those rings is in-thread), the 2 warps of a CTA own 32 rings of the same
//            32 degrees, summed through shared memory; per-CTA partials over 32-ring blocks are
//            summed in a fixed order.
// Small CTAs (64 threads) keep the work per CTA small: the chains' lengths grow with the degree,
// and fewer, larger CTAs left the GPU idle behind the high-degree ones (measured).
// Chains of one lane share lambda_m (inverse) or are fed from lane-uniform shared-memory values
// (forward: lambda_m and g_m per ring); their starting values are computed before the sweep and
// held in the chain registers until the recursion reaches m = l.
#include <cuda_runtime.h>

#include "theta_common.cuh"

namespace s2gb {

namespace {
using namespace theta;

constexpr int kIW = 2;         // inverse: warps per CTA
constexpr int kIK = 16;        // inverse: degrees (chains) per lane
constexpr int kIL = kIW * kIK; // inverse: degrees per CTA
constexpr int kFW = 2;         // forward: warps per CTA
constexpr int kFT = 16;        // forward: rings (chains) per lane
constexpr int kFR = kFW * kFT; // forward: rings per CTA
constexpr int kCh = 8;         // inverse: orders per staged chunk
constexpr int kChF = 4;        // forward: orders per staged chunk

// Ring seen from pi - b (chain B): same v, the other hemisphere, sin/cos of the half angle swapped.
__device__ __forceinline__ RingData reflect_ring(const RingData& r) {
  RingData o = r;
  o.ls_hi = r.lc_hi; o.ls_lo = r.lc_lo;
  o.lc_hi = r.ls_hi; o.lc_lo = r.ls_lo;
  o.north = !r.north;
  o.pole = r.pole == 1 ? 2 : (r.pole == 2 ? 1 : 0);
  return o;
}

// lambda_m = (n - m cos b) / sin b from v and 1/sin b
__device__ __forceinline__ double lambda_m(int m, int n, double v, double csc, bool north) {
  const double dm = (double)m;
  return (north ? fma(dm, v, (double)(n - m)) : fma(-dm, v, (double)(n + m))) * csc;
}

// one step m -> m-1 of a chain: (x, y) = (d_m, d_{m+1}) -> (d_{m-1}, d_m)
__device__ __forceinline__ void mstep(double& x, double& y, double lam, double2 ab) {
  const double xn = fma(lam * ab.x, x, -(ab.y * y));
  y = x;
  x = xn;
}

// ------------------------------------------------------------------------------------------
// Inverse.  Grid: x = tile of 32 rings, y = degree group (32 degrees, highest first), z = n index
// x batch groups of NB signals.  part layout: [group][S][2L-1 (m + L - 1)][nint (ring - ring0)].
// ------------------------------------------------------------------------------------------
template <int NB, bool PAIR>
struct InvSmem {
  static constexpr int NBX = PAIR ? 2 * NB : NB;
  double2 h[kCh][kIL][NBX];      // h_{l,m} scale_l (sign of chain B / the -m partner folded in)
  double2 ab[kCh][kIL];          // (a_{m-1}, a_{m-1}/a_m)
  double2 red[2][kIW][32][NBX];  // per-warp partials of one step
};

template <int NB, bool PAIR, bool REFL>
__device__ __forceinline__ void inverse_sweep(const InvArgs& a, const MrecArgs& q, InvSmem<NB, PAIR>& sm,
                                              int ni, int n, int sig0, int g, int l0, int ltop,
                                              int t, bool tok, const RingData& rd0, double csc,
                                              int mstar, int mlow) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  const int L = a.L, T = 2 * L - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lw = l0 + warp * kIK;                  // this warp's degrees [lw, lw + kIK)
  const int an = n < 0 ? -n : n;
  const RingData rd = REFL ? reflect_ring(rd0) : rd0;
  const bool north = rd.north;
  const double v = rd.v;
  // outputs of this lane: m >= mstar (chain A) or m' >= 1 - mstar (chain B, m = -m')
  const int mvalid = REFL ? 1 - mstar : mstar;

  double x[kIK], y[kIK];
  int E[kIK];
#pragma unroll
  for (int k = 0; k < kIK; ++k) {
    const int l = lw + k;
    y[k] = 0.0;
    if (tok && l >= an && l < L) {
      seed_value(a.seed[(size_t)ni * T + l + L - 1], rd, x[k], E[k]);   // d^l_{l,n}, Eq. initial_values
    } else {
      x[k] = 0.0; E[k] = 0;
    }
  }
  const long long nsigs = (long long)a.nsig * a.nN;
  double2* part = reinterpret_cast<double2*>(q.part) + (size_t)g * nsigs * T * q.nint;
  int buf = 0;
  unsigned live = 0;
  for (int mc = ltop; mc >= mlow; mc -= kCh) {
    // stage the coefficients and h for the orders mc, mc-1, ..., mc-kCh+1
    __syncthreads();
    for (int idx = threadIdx.x; idx < kCh * kIL * NBX; idx += blockDim.x) {
      const int b = idx % NBX, d = (idx / NBX) % kIL, j = idx / (NBX * kIL);
      const int l = l0 + d, mm = mc - j;
      const int bb = PAIR ? (b % NB) : b;
      const bool partner = PAIR && b >= NB;
      const int mo = REFL ? -mm : (partner ? -mm : mm);    // order of the output
      const int sig = sig0 + bb;
      double2 h = make_double2(0.0, 0.0);
      if (sig < a.nsig && l < L && l >= an && mm >= 0 - l && mm <= l && !(partner && mm <= 0)) {
        h = reinterpret_cast<const double2*>(a.flm)[((size_t)(sig * a.nN + ni) * L + l) * a.flm_ld + mo + a.flm_c0];
        double s = a.scale[(size_t)ni * L + l];
        if (REFL && ((l + n) & 1)) s = -s;                   // (-1)^{l+n}
        if (partner && (mm & 1)) s = -s;                     // (-1)^m
        h.x *= s; h.y *= s;
      }
      sm.h[j][d][b] = h;
    }
    for (int idx = threadIdx.x; idx < kCh * kIL; idx += blockDim.x) {
      const int d = idx % kIL, j = idx / kIL;
      const int l = l0 + d, mm = mc - j;
      sm.ab[j][d] = (l < L && mm <= l && mm > -l) ? q.ab[(size_t)l * T + mm + L - 1] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int jend = min(kCh, mc - mlow + 1);
    for (int j = 0; j < jend; ++j) {
      const int m = mc - j;
      if (((ltop - m) & 7) == 0) {
        live = 0;
#pragma unroll
        for (int k = 0; k < kIK; ++k) live |= (__any_sync(0xffffffffu, E[k] == 0 && x[k] != 0.0) ? 1u : 0u) << k;
      }
      double2 acc[NBX];
#pragma unroll
      for (int b = 0; b < NBX; ++b) acc[b] = make_double2(0.0, 0.0);
      const bool outok = tok && m >= mvalid;
      if (lw <= ltop && m <= lw + kIK - 1) {           // some chain of this warp has started
#pragma unroll
        for (int k = 0; k < kIK; ++k) {
          if (((live >> k) & 1u) && m <= lw + k) {
            const double xl = (E[k] == 0 && outok) ? x[k] : 0.0;
#pragma unroll
            for (int b = 0; b < NBX; ++b) {
              const double2 h = sm.h[j][warp * kIK + k][b];
              acc[b].x = fma(xl, h.x, acc[b].x);
              acc[b].y = fma(xl, h.y, acc[b].y);
            }
          }
        }
        if (m > mlow) {
          const double lam = lambda_m(m, n, v, csc, north);
#pragma unroll
          for (int k = 0; k < kIK; ++k)
            if (m <= lw + k) mstep(x[k], y[k], lam, sm.ab[j][warp * kIK + k]);
        }
        if (((ltop - m) & 7) == 7) {
#pragma unroll
          for (int k = 0; k < kIK; ++k) renorm(x[k], y[k], E[k]);
        }
      }
      // fixed-order sum over the warps, one partial per CTA
#pragma unroll
      for (int b = 0; b < NBX; ++b) sm.red[buf][warp][lane][b] = acc[b];
      __syncthreads();
      for (int idx = threadIdx.x; idx < 32 * NBX; idx += blockDim.x) {
        // idx % 32 is this thread's lane, so the output ring is the lane's own ring (every warp
        // holds the same 32 rings)
        const int ln = idx % 32, b = idx / 32;
        const int bb = PAIR ? (b % NB) : b;
        const bool partner = PAIR && b >= NB;
        const int mo = REFL ? -m : (partner ? -m : m);
        // this ring's output: chain A for m >= mstar, chain B for m <= mstar - 1
        const bool own = REFL ? (m >= 1 - mstar) : (m >= mstar);
        if (tok && sig0 + bb < a.nsig && own && !(partner && m <= 0)) {
          double2 s = sm.red[buf][0][ln][b];
          for (int w = 1; w < kIW; ++w) {
            const double2 r = sm.red[buf][w][ln][b];
            s.x += r.x; s.y += r.y;
          }
          part[((size_t)((sig0 + bb) * a.nN + ni) * T + mo + L - 1) * q.nint + (t - a.ring0)] = s;
        }
      }
      buf ^= 1;
    }
  }
}

template <int NB, bool PAIR>
__global__ void __launch_bounds__(kIW * 32) mrec_inverse_kernel(InvArgs a, MrecArgs q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  InvSmem<NB, PAIR>& sm = *reinterpret_cast<InvSmem<NB, PAIR>*>(smem_raw);
  const int L = a.L;
  const int lane = threadIdx.x & 31;
  const int g = gridDim.y - 1 - blockIdx.y;          // highest degrees first
  const int l0 = g * kIL;
  const int ltop = min(L - 1, l0 + kIL - 1);
  const int nbg = (a.nsig + NB - 1) / NB;
  const int ni = blockIdx.z / nbg, sig0 = (blockIdx.z % nbg) * NB;
  const int n = q.n_of[ni];
  if (ltop < (n < 0 ? -n : n)) return;               // no degree l >= |n| here
  const int t = a.ring0 + blockIdx.x * 32 + lane;
  const bool tok = t < a.nring;
  RingData rd{};
  double csc = 0.0;
  if (tok) { rd = a.ring[t]; csc = q.csc[t]; }
  else { rd.north = 1; }
  const double cb = rd.north ? 1.0 - rd.v : rd.v - 1.0;
  const int mstar = PAIR ? 0 : min(ltop, max(-ltop, (int)rint((double)n * cb)));
  // the CTA's sweeps run down to the lowest order any of its lanes needs
  const int big = 1 << 30;
  const int mlow1 = PAIR ? 0 : __reduce_min_sync(0xffffffffu, tok ? mstar : big);
  inverse_sweep<NB, PAIR, false>(a, q, sm, ni, n, sig0, g, l0, ltop, t, tok, rd, csc, mstar,
                                 min(mlow1, ltop));
  if (!PAIR) {
    const int mlow2 = __reduce_min_sync(0xffffffffu, tok ? 1 - mstar : big);
    if (mlow2 <= ltop)
      inverse_sweep<NB, PAIR, true>(a, q, sm, ni, n, sig0, g, l0, ltop, t, tok, rd, csc, mstar, mlow2);
  }
}

// ------------------------------------------------------------------------------------------
// Forward.  Grid: x = degree group (32 degrees, highest first), y = block of 32 rings, z = n
// index x batch groups.  part layout: [ring block][S][L][2L-1] (the flm layout).
// ------------------------------------------------------------------------------------------
template <int NB, bool PAIR>
struct FwdSmem {
  static constexpr int NBX = PAIR ? 2 * NB : NB;
  double2 gv[kChF][kFR][NBX];     // g_m(t) (times the ring weight; the -m partner with (-1)^m)
  double lam[kChF][kFR];          // lambda_m(t)
  double2 ab[kChF][32];           // (a_{m-1}, a_{m-1}/a_m) of the 32 degrees
  double2 red[2][kFW][32][NBX];
  int mstar[kFR];
};

template <int NB, bool PAIR, bool REFL>
__device__ __forceinline__ void forward_sweep(const FwdArgs& a, const MrecArgs& q, FwdSmem<NB, PAIR>& sm,
                                              int ni, int n, int sig0, int gr, int lg0, int ltop,
                                              int r0, int mlow) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  const int L = a.L, T = 2 * L - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = lg0 + lane;                          // this lane's degree
  const int an = n < 0 ? -n : n;
  const bool lok = l < L && l >= an;
  const int rend = a.row0 + a.nrows;

  double x[kFT], y[kFT];
  int E[kFT];
#pragma unroll
  for (int i = 0; i < kFT; ++i) {
    const int t = r0 + warp * kFT + i;
    y[i] = 0.0;
    if (lok && t < rend) {
      RingData rd = a.ring[t];
      if (REFL) rd = reflect_ring(rd);
      seed_value(a.seed[(size_t)ni * T + l + L - 1], rd, x[i], E[i]);
    } else {
      x[i] = 0.0; E[i] = 0;
    }
  }
  const long long nsigs = (long long)a.nsig * a.nN;
  double2* part = reinterpret_cast<double2*>(q.part) + (size_t)gr * nsigs * L * T;
  int buf = 0;
  unsigned live = 0;
  for (int mc = ltop; mc >= mlow; mc -= kChF) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kChF * kFR * NBX; idx += blockDim.x) {
      const int b = idx % NBX, rr = (idx / NBX) % kFR, j = idx / (NBX * kFR);
      const int t = r0 + rr, mm = mc - j;
      const int bb = PAIR ? (b % NB) : b;
      const bool partner = PAIR && b >= NB;
      const int mo = REFL ? -mm : (partner ? -mm : mm);
      const int sig = sig0 + bb;
      double2 gval = make_double2(0.0, 0.0);
      if (sig < a.nsig && t < rend && mo > -L && mo < L && !(partner && mm <= 0)) {
        const long long col = a.m_mod ? (mo >= 0 ? mo : mo + a.mmod) : (long long)(mo + L - 1);
        gval = reinterpret_cast<const double2*>(a.g)[(size_t)(sig * a.nN + ni) * a.s_sig + (size_t)t * a.s_t + col * a.s_m];
        double w = a.use_nu ? a.nu[t] : 1.0;
        if (partner && (mm & 1)) w = -w;                    // (-1)^m
        gval.x *= w; gval.y *= w;
      }
      sm.gv[j][rr][b] = gval;
    }
    for (int idx = threadIdx.x; idx < kChF * kFR; idx += blockDim.x) {
      const int rr = idx % kFR, j = idx / kFR;
      const int t = r0 + rr, mm = mc - j;
      double lam = 0.0;
      if (t < rend) {
        const RingData rd = a.ring[t];
        lam = lambda_m(mm, n, rd.v, q.csc[t], REFL ? !rd.north : (bool)rd.north);
      }
      sm.lam[j][rr] = lam;
    }
    for (int idx = threadIdx.x; idx < kChF * 32; idx += blockDim.x) {
      const int d = idx % 32, j = idx / 32;
      const int ll = lg0 + d, mm = mc - j;
      sm.ab[j][d] = (ll < L && mm <= ll && mm > -ll) ? q.ab[(size_t)ll * T + mm + L - 1] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int jend = min(kChF, mc - mlow + 1);
    for (int j = 0; j < jend; ++j) {
      const int m = mc - j;
      if (((ltop - m) & 7) == 0) {
        live = 0;
#pragma unroll
        for (int i = 0; i < kFT; ++i) live |= (__any_sync(0xffffffffu, E[i] == 0 && x[i] != 0.0) ? 1u : 0u) << i;
      }
      double2 p[NBX];
#pragma unroll
      for (int b = 0; b < NBX; ++b) p[b] = make_double2(0.0, 0.0);
      const bool started = m <= l;
#pragma unroll
      for (int i = 0; i < kFT; ++i) {
        const int rr = warp * kFT + i;
        const int ms = sm.mstar[rr];
        const bool valid = REFL ? (m >= 1 - ms) : (m >= ms);
        if (((live >> i) & 1u) && valid) {
          const double xl = (E[i] == 0 && started) ? x[i] : 0.0;
#pragma unroll
          for (int b = 0; b < NBX; ++b) {
            const double2 gv = sm.gv[j][rr][b];
            p[b].x = fma(xl, gv.x, p[b].x);
            p[b].y = fma(xl, gv.y, p[b].y);
          }
        }
      }
      if (m > mlow) {
        const double2 ab = sm.ab[j][lane];
#pragma unroll
        for (int i = 0; i < kFT; ++i)
          if (started) mstep(x[i], y[i], sm.lam[j][warp * kFT + i], ab);
      }
      if (((ltop - m) & 7) == 7) {
#pragma unroll
        for (int i = 0; i < kFT; ++i) renorm(x[i], y[i], E[i]);
      }
#pragma unroll
      for (int b = 0; b < NBX; ++b) sm.red[buf][warp][lane][b] = p[b];
      __syncthreads();
      for (int idx = threadIdx.x; idx < 32 * NBX; idx += blockDim.x) {
        const int ln = idx % 32, b = idx / 32;
        const int bb = PAIR ? (b % NB) : b;
        const bool partner = PAIR && b >= NB;
        const int ll = lg0 + ln;
        const int mo = REFL ? -m : (partner ? -m : m);
        const int amo = mo < 0 ? -mo : mo;
        if (ll < L && ll >= an && amo <= ll && sig0 + bb < a.nsig && !(partner && m <= 0)) {
          double2 s = sm.red[buf][0][ln][b];
          for (int w = 1; w < kFW; ++w) {
            const double2 r = sm.red[buf][w][ln][b];
            s.x += r.x; s.y += r.y;
          }
          double sc = a.scale[(size_t)ni * L + ll];                // per-degree factor
          if (REFL && ((ll + n) & 1)) sc = -sc;                     // (-1)^{l+n}
          s.x *= sc; s.y *= sc;
          double2* o = part + ((size_t)((sig0 + bb) * a.nN + ni) * L + ll) * T + mo + L - 1;
          // chain B's orders overlap chain A's where the rings' split points differ: add there
          if (REFL && mo >= q.mlow1) { const double2 prev = *o; s.x += prev.x; s.y += prev.y; }
          *o = s;
        }
      }
      buf ^= 1;
    }
  }
}

template <int NB, bool PAIR>
__global__ void __launch_bounds__(kFW * 32) mrec_forward_kernel(FwdArgs a, MrecArgs q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FwdSmem<NB, PAIR>& sm = *reinterpret_cast<FwdSmem<NB, PAIR>*>(smem_raw);
  const int L = a.L;
  const int lg0 = (gridDim.x - 1 - blockIdx.x) * 32;  // highest degrees first
  const int ltop = min(L - 1, lg0 + 31);
  const int gr = blockIdx.y;
  const int r0 = a.row0 + gr * kFR;
  const int rend = a.row0 + a.nrows;
  const int nbg = (a.nsig + NB - 1) / NB;
  const int ni = blockIdx.z / nbg, sig0 = (blockIdx.z % nbg) * NB;
  const int n = q.n_of[ni];
  const int an = n < 0 ? -n : n;
  // every part must hold this CTA's degrees even if all are below |n|: write nothing there (the sum
  // masks l < |n|), so only the sweeps need |n| <= ltop
  if (ltop < an) return;
  // split points m* of the CTA's rings (lane-uniform values for the chains)
  int lo = 1 << 30, hi = -(1 << 30);
  for (int rr = threadIdx.x; rr < kFR; rr += blockDim.x) {
    const int t = r0 + rr;
    int ms = 0;
    if (t < rend) {
      const RingData rd = a.ring[t];
      const double cb = rd.north ? 1.0 - rd.v : rd.v - 1.0;
      ms = PAIR ? 0 : min(ltop, max(-ltop, (int)rint((double)n * cb)));
      lo = min(lo, ms);
      hi = max(hi, ms);
    }
    sm.mstar[rr] = ms;
  }
  // CTA-wide min / max of the split points (fixed values, any reduction order)
  __shared__ int mm_red[2];
  if (threadIdx.x == 0) { mm_red[0] = 1 << 30; mm_red[1] = -(1 << 30); }
  __syncthreads();
  atomicMin(&mm_red[0], lo);
  atomicMax(&mm_red[1], hi);
  __syncthreads();
  const int mlow1 = PAIR ? 0 : mm_red[0];
  MrecArgs qq = q;
  qq.mlow1 = mlow1;
  forward_sweep<NB, PAIR, false>(a, qq, sm, ni, n, sig0, gr, lg0, ltop, r0, mlow1);
  if (!PAIR) {
    const int mlow2 = 1 - mm_red[1];
    if (mlow2 <= ltop) forward_sweep<NB, PAIR, true>(a, qq, sm, ni, n, sig0, gr, lg0, ltop, r0, mlow2);
  }
}

// ftilde (strides of the output) = fixed-order sum over the degree groups that reach |m|
__global__ void mrec_sum_inverse_kernel(InvArgs a, MrecArgs q, int ngroups) {
  const int L = a.L, T = 2 * L - 1;
  const long long nsigs = (long long)a.nsig * a.nN;
  const size_t total = (size_t)nsigs * T * q.nint;
  const double2* part = reinterpret_cast<const double2*>(q.part);
  const size_t gstride = (size_t)nsigs * T * q.nint;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int tr = (int)(idx % q.nint);
    const int mi = (int)((idx / q.nint) % T);
    const size_t s = idx / ((size_t)q.nint * T);
    const int m = mi - (L - 1);
    const int am = m < 0 ? -m : m;
    if (am < q.mlo || am >= q.mhi) continue;
    const int n = q.n_of[s % a.nN];
    const int an = n < 0 ? -n : n;
    const int need = am > an ? am : an;              // groups whose top degree reaches max(|m|, |n|)
    double2 acc = make_double2(0.0, 0.0);
    for (int g = 0; g < ngroups; ++g) {
      if (min(L - 1, g * kIL + kIL - 1) < need) continue;
      const double2 v = part[g * gstride + idx];
      acc.x += v.x; acc.y += v.y;
    }
    const long long col = a.m_mod ? (m >= 0 ? m : m + a.mmod) : (long long)(m + L - 1);
    reinterpret_cast<double2*>(a.out)[s * a.s_sig + (size_t)(a.ring0 + tr) * a.s_t + col * a.s_m] = acc;
  }
}

// flm = fixed-order sum over the ring blocks; 0 where |m| > l or l < |n|
__global__ void mrec_sum_forward_kernel(FwdArgs a, MrecArgs q, int ngroups) {
  const int L = a.L, T = 2 * L - 1;
  const long long nsigs = (long long)a.nsig * a.nN;
  const size_t total = (size_t)nsigs * L * T;
  const double2* part = reinterpret_cast<const double2*>(q.part);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int mi = (int)(idx % T);
    const int l = (int)((idx / T) % L);
    const size_t s = idx / ((size_t)T * L);
    const int m = mi - (L - 1);
    const int am = m < 0 ? -m : m;
    if (am < q.mlo || am >= q.mhi) continue;
    const int n = q.n_of[s % a.nN];
    const int an = n < 0 ? -n : n;
    double2 acc = make_double2(0.0, 0.0);
    if (am <= l && an <= l) {
      for (int g = 0; g < ngroups; ++g) {
        const double2 v = part[(size_t)g * total + idx];
        acc.x += v.x; acc.y += v.y;
      }
    }
    reinterpret_cast<double2*>(a.flm)[(s * L + l) * a.flm_ld + m + a.flm_c0] = acc;
  }
}

inline unsigned sum_grid(size_t n) {
  size_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g ? g : 1);
}

template <int NB, bool PAIR>
cudaError_t launch_inv_m(const Plan& p, const InvArgs& a, const MrecArgs& q, cudaStream_t st) {
  const int nt = a.nring - a.ring0;
  if (nt > 0) {
    const size_t smem = sizeof(InvSmem<NB, PAIR>);
    auto kern = mrec_inverse_kernel<NB, PAIR>;
    cudaError_t e = set_dynamic_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((nt + 31) / 32), (unsigned)((a.L + kIL - 1) / kIL),
              (unsigned)(a.nN * ((a.nsig + NB - 1) / NB)));
    kern<<<grid, kIW * 32, smem, st>>>(a, q);
    if ((e = launched()) != cudaSuccess) return e;
  }
  const size_t n = (size_t)a.nsig * a.nN * (2 * a.L - 1) * q.nint;
  mrec_sum_inverse_kernel<<<sum_grid(n), 256, 0, st>>>(a, q, nt > 0 ? (a.L + kIL - 1) / kIL : 0);
  return launched();
}

template <int NB, bool PAIR>
cudaError_t launch_fwd_m(const Plan& p, const FwdArgs& a, const MrecArgs& q, cudaStream_t st) {
  const int nr = a.nrows;
  const int nblocks = (nr + kFR - 1) / kFR;
  if (nr > 0) {
    const size_t smem = sizeof(FwdSmem<NB, PAIR>);
    auto kern = mrec_forward_kernel<NB, PAIR>;
    cudaError_t e = set_dynamic_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.L + 31) / 32), (unsigned)nblocks, (unsigned)(a.nN * ((a.nsig + NB - 1) / NB)));
    kern<<<grid, kFW * 32, smem, st>>>(a, q);
    if ((e = launched()) != cudaSuccess) return e;
  }
  const size_t n = (size_t)a.nsig * a.nN * a.L * (2 * a.L - 1);
  mrec_sum_forward_kernel<<<sum_grid(n), 256, 0, st>>>(a, q, nr > 0 ? nblocks : 0);
  return launched();
}

MrecArgs mrec_args(const Plan& p, void* part, int rank0, int nrank) {
  MrecArgs q{};
  q.ab = reinterpret_cast<const double2*>(p.mrec_ab);
  q.csc = p.csc;
  q.n_of = p.n_of;
  q.part = part;
  q.nint = p.nint;
  q.mlo = (rank0 + 1) / 2;
  q.mhi = (rank0 + nrank + 1) / 2;
  q.mlow1 = 0;
  return q;
}

}  // namespace

size_t mrec_part_bytes(const Plan& p, int batch) {
  const size_t S = (size_t)batch * p.nN;
  const size_t T = p.T;
  const size_t gi = (size_t)(p.L + kIL - 1) / kIL, gf = (size_t)(p.nint + kFR - 1) / kFR;
  const size_t inv = gi * S * T * (size_t)p.nint, fwd = gf * S * (size_t)p.L * T;
  return 16 * (inv > fwd ? inv : fwd);
}

// n = 0 pairs the orders m and -m (spin-0 sphere plans); Wigner plans run every n unpaired
bool mrec_paired(const Plan& p) { return !p.wigner && !p.real && p.spin == 0; }

cudaError_t launch_theta_inverse_mrec(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (!a.mpart && p.nint > 0) return cudaErrorInvalidValue;   // no rings: nothing is written there
  const MrecArgs q = mrec_args(p, a.mpart, a.rank0, a.nrank);
  if (mrec_paired(p)) {
    if (a.nsig >= 2) return launch_inv_m<2, true>(p, a, q, st);
    return launch_inv_m<1, true>(p, a, q, st);
  }
  if (a.nsig >= 4) return launch_inv_m<4, false>(p, a, q, st);
  if (a.nsig >= 2) return launch_inv_m<2, false>(p, a, q, st);
  return launch_inv_m<1, false>(p, a, q, st);
}

cudaError_t launch_theta_forward_mrec(const Plan& p, const FwdArgs& a, cudaStream_t st) {
  if (!a.mpart && p.nint > 0) return cudaErrorInvalidValue;
  const MrecArgs q = mrec_args(p, a.mpart, a.rank0, a.nrank);
  FwdArgs b = a;
  b.row0 = p.ring0;
  b.nrows = p.nint;
  if (mrec_paired(p)) {
    if (a.nsig >= 2) return launch_fwd_m<2, true>(p, b, q, st);
    return launch_fwd_m<1, true>(p, b, q, st);
  }
  if (a.nsig >= 4) return launch_fwd_m<4, false>(p, b, q, st);
  if (a.nsig >= 2) return launch_fwd_m<2, false>(p, b, q, st);
  return launch_fwd_m<1, false>(p, b, q, st);
}

}  // namespace s2gb
