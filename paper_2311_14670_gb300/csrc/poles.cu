// Pole rings: theta = 0 and pi on MWSS sampling, and theta = pi on MW sampling when the theta stage
// runs the order recursion (whose lambda_m = (n - m cos b)/sin b is undefined there).  There the
// Wigner d-functions are Kronecker deltas (Sec. 3.3):
//     d^l_{mn}(0) = delta_{m,n},        d^l_{mn}(pi) = (-1)^{l-n} delta_{m,-n},
// so each pole ring couples one order to the coefficients and the three-term recursion is not
// needed there.  The recursion kernels run over the other rings only, and these kernels supply the
// poles exactly:
//   inverse-shaped:  ftilde_m(pole) = [m = m*] sum_{l >= |n|} scale_l flm_{l,m*} sgn_l,
//   forward-shaped:  flm_{l,m*} += scale_l w_pole sgn_l g_{m*}(pole)      (after the interior sum),
// with m* = n, sgn_l = 1 at theta = 0 and m* = -n, sgn_l = (-1)^{l-n} at theta = pi, and w_pole the
// ring weight (1 for the self-reflected rings theta = 0, pi of MW and MWSS, or 1 in the unweighted
// adjoint).  Sums run in a
// fixed order (deterministic).  Data are complex128 or complex64 (accumulated in float64).
#include <cuda_runtime.h>

#include "s2gb_internal.h"

namespace s2gb {

namespace {

template <typename C>
struct Real;
template <>
struct Real<double2> { using type = double; };
template <>
struct Real<float2> { using type = float; };

constexpr int kPoleThreads = 256;

// Grid: x = signal index s = sig * nN + ni, y = pole (0: theta = 0 at ring pn; 1: theta = pi at
// ring ps; a negative ring index means the plan has no such ring).  Writes the pole ring of every
// order with |m| in [mlo, mhi).
template <typename C>
__global__ void __launch_bounds__(kPoleThreads) pole_inverse_kernel(InvArgs a, const int* __restrict__ n_of,
                                                                    int mlo, int mhi, int pn, int ps) {
  using Rl = typename Real<C>::type;
  __shared__ double red[2][kPoleThreads / 32];
  __shared__ double2 val;
  const int L = a.L;
  const int s = blockIdx.x, pole = blockIdx.y;
  const int t = pole ? ps : pn;
  if (t < 0) return;
  const int ni = s % a.nN;
  const int n = n_of[ni];
  const int ms = pole ? -n : n;
  const int am = ms < 0 ? -ms : ms;
  const bool own = am >= mlo && am < mhi;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (own) {
    double vr = 0.0, vi = 0.0;
    const double* scale = a.scale + (size_t)ni * L;
    const C* flm = reinterpret_cast<const C*>(a.flm) + (size_t)s * L * a.flm_ld + ms + a.flm_c0;
    for (int l = am + threadIdx.x; l < L; l += blockDim.x) {
      const C h = flm[(size_t)l * a.flm_ld];
      const double w = (pole && ((l - n) & 1)) ? -scale[l] : scale[l];
      vr = fma(w, (double)h.x, vr);
      vi = fma(w, (double)h.y, vi);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      vr += __shfl_down_sync(0xffffffffu, vr, off);
      vi += __shfl_down_sync(0xffffffffu, vi, off);
    }
    if (lane == 0) { red[0][warp] = vr; red[1][warp] = vi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0, ti = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tr += red[0][w]; ti += red[1][w]; }
      val = make_double2(tr, ti);
    }
  }
  __syncthreads();
  C* out = reinterpret_cast<C*>(a.out) + (size_t)s * a.s_sig + (size_t)t * a.s_t;
  for (int q = threadIdx.x; q < 2 * L - 1; q += blockDim.x) {
    const int m = q - (L - 1);
    const int aq = m < 0 ? -m : m;
    if (aq < mlo || aq >= mhi) continue;
    const long long col = a.m_mod ? (m >= 0 ? m : m + a.mmod) : (long long)(m + L - 1);
    C o;
    o.x = (m == ms) ? (Rl)val.x : (Rl)0;
    o.y = (m == ms) ? (Rl)val.y : (Rl)0;
    out[col * a.s_m] = o;
  }
}

// One thread per (signal index s, degree l): adds the two pole terms, theta = 0 first.
template <typename C>
__global__ void pole_forward_kernel(FwdArgs a, const int* __restrict__ n_of, int mlo, int mhi, int pn, int ps) {
  using Rl = typename Real<C>::type;
  const int L = a.L;
  const size_t total = (size_t)a.nsig * a.nN * L;
  C* flm = reinterpret_cast<C*>(a.flm);
  const C* g = reinterpret_cast<const C*>(a.g);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx % L);
    const size_t s = idx / L;
    const int ni = (int)(s % a.nN);
    const int n = n_of[ni];
    const int an = n < 0 ? -n : n;
    if (l < an || an < mlo || an >= mhi) continue;
    const double sc = a.scale[(size_t)ni * L + l];
    for (int pole = 0; pole < 2; ++pole) {
      const int t = pole ? ps : pn;
      if (t < 0) continue;
      const int m = pole ? -n : n;
      const long long col = a.m_mod ? (m >= 0 ? m : m + a.mmod) : (long long)(m + L - 1);
      const C gv = g[s * a.s_sig + (size_t)t * a.s_t + col * a.s_m];
      double w = (a.use_nu ? a.nu[t] : 1.0) * sc;
      if (pole && ((l - n) & 1)) w = -w;
      C* o = flm + (s * L + l) * a.flm_ld + m + a.flm_c0;
      C v = *o;
      v.x = (Rl)fma(w, (double)gv.x, (double)v.x);
      v.y = (Rl)fma(w, (double)gv.y, (double)v.y);
      *o = v;
    }
  }
}

// |m| range of the m-ranks [rank0, rank0 + nrank) of the 0, -1, 1, -2, 2, ... order
void rank_orders(int rank0, int nrank, int& mlo, int& mhi) {
  mlo = (rank0 + 1) / 2;
  mhi = (rank0 + nrank + 1) / 2;
}

}  // namespace

cudaError_t launch_pole_inverse(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (a.mpos) return cudaErrorInvalidValue;         // MWSS plans are complex-signal plans
  int mlo, mhi;
  rank_orders(a.rank0, a.nrank, mlo, mhi);
  dim3 grid((unsigned)(a.nsig * a.nN), 2);
  if (p.precision == S2GB_FP64)
    pole_inverse_kernel<double2><<<grid, kPoleThreads, 0, st>>>(a, p.n_of, mlo, mhi, p.pole_n, p.pole_s);
  else
    pole_inverse_kernel<float2><<<grid, kPoleThreads, 0, st>>>(a, p.n_of, mlo, mhi, p.pole_n, p.pole_s);
  return launched();
}

cudaError_t launch_pole_forward(const Plan& p, const FwdArgs& a, cudaStream_t st) {
  if (a.mpos) return cudaErrorInvalidValue;
  int mlo, mhi;
  rank_orders(a.rank0, a.nrank, mlo, mhi);
  const size_t n = (size_t)a.nsig * a.nN * a.L;
  const unsigned blocks = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (p.precision == S2GB_FP64)
    pole_forward_kernel<double2><<<blocks, 256, 0, st>>>(a, p.n_of, mlo, mhi, p.pole_n, p.pole_s);
  else
    pole_forward_kernel<float2><<<blocks, 256, 0, st>>>(a, p.n_of, mlo, mhi, p.pole_n, p.pole_s);
  return launched();
}

}  // namespace s2gb
