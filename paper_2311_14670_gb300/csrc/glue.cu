// Memory-bound glue between the FFT stages of the transforms: the theta torus extension of the MW
// and MWSS grids (Sec. 4.2.2) and its adjoint, Fourier-domain zero padding and truncation, the
// fine-grid weights of the forward quadrature, ring weights (DH), and the gamma-axis reordering of
// the Wigner transform.
// Every kernel is a grid-stride loop over its output with one thread per complex element.
#include <cuda_runtime.h>

#include "s2gb_internal.h"

namespace s2gb {

namespace {

template <typename C>
struct RealOf;
template <>
struct RealOf<double2> { using type = double; };
template <>
struct RealOf<float2> { using type = float; };

inline unsigned grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g ? g : 1);
}

// Theta-torus geometry of the MW and MWSS grids (Sec. 4.2.2).  Torus point t' < TS is ring t'
// for t' < R and the reflection theta -> 2 pi - theta of ring refl(t') = O - t' otherwise, with
// O = 2L-2 (MW, TS = 2L-1, R = L) or O = 2L (MWSS, TS = 2L, R = L+1).  Rings that are their own
// reflection (theta = pi on MW; theta = 0 and pi on MWSS) have self_ring() true.
struct Torus {
  int L, R, TS, O;
  __device__ bool self_ring(int t) const { return (t == O - t) || (TS == 2 * L && t == 0); }
};

// G[s][r][t'] (t' < TS) from F[s][t][k] (t < R): the ring value for t' < R, sigma times the
// reflected ring's value beyond, and (1+sigma)/2 F on a self-reflected ring; sigma = (-1)^{m-n}.
// Row r of G is order m = r - mo (MR rows); F has rows of FW columns with column k = m mod FW
// (complex signals: MR = T, mo = L-1, FW = P; real signals, m >= 0 only: MR = FW = L, mo = 0).
template <typename C>
__global__ void extend_kernel(const C* __restrict__ F, C* __restrict__ G, int S, Torus tor, int nN,
                              const int* __restrict__ n_of, int MR, int mo, int FW) {
  const int TS = tor.TS, R = tor.R;
  const size_t total = (size_t)S * MR * TS;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int tp = (int)(idx % TS);
    const int r = (int)((idx / TS) % MR);
    const int s = (int)(idx / ((size_t)TS * MR));
    const int m = r - mo;
    const int k = m >= 0 ? m : m + FW;
    const int n = n_of[s % nN];
    const bool odd = ((m - n) & 1) != 0;
    C out;
    if (tp < R) {
      const C v = F[((size_t)s * R + tp) * FW + k];
      out = (tor.self_ring(tp) && odd) ? C{0, 0} : v;
    } else {
      const C v = F[((size_t)s * R + (tor.O - tp)) * FW + k];
      out = odd ? C{-v.x, -v.y} : v;
    }
    G[idx] = out;
  }
}

// Adjoint of extend_kernel: F[s][t][k] = G[s][r][t] + sigma G[s][r][O-t] on rings with a
// reflection, (1+sigma)/2 G[s][r][t] on self-reflected rings, for every column k of F (FW columns;
// a column no order owns -- k = L on MWSS -- is 0).
template <typename C>
__global__ void extend_adjoint_kernel(const C* __restrict__ G, C* __restrict__ F, int S, Torus tor, int nN,
                                      const int* __restrict__ n_of, int MR, int mo, int FW) {
  const int TS = tor.TS, R = tor.R, L = tor.L;
  const size_t total = (size_t)S * R * FW;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % FW);
    const int t = (int)((idx / FW) % R);
    const int s = (int)(idx / ((size_t)FW * R));
    int m;
    if (mo == 0) m = k;                          // real signals: column k is order m = k
    else if (k <= L - 1) m = k;
    else if (k >= FW - (L - 1)) m = k - FW;
    else { F[idx] = C{0, 0}; continue; }         // MWSS: the phi frequency L has no order
    const int r = m + mo;
    const int n = n_of[s % nN];
    const bool odd = ((m - n) & 1) != 0;
    const C* row = G + ((size_t)s * MR + r) * TS;
    C out;
    if (tor.self_ring(t)) {
      out = odd ? C{0, 0} : row[t];
    } else {
      const C a = row[t], b = row[tor.O - t];
      out = odd ? C{a.x - b.x, a.y - b.y} : C{a.x + b.x, a.y + b.y};
    }
    F[idx] = out;
  }
}

// Y[r][q] (q < NF) = X[r][k mod TS] for the frequency k = q (q <= L-1) or q - NF (q >= NF-L+1).
template <typename C>
__global__ void pad_kernel(const C* __restrict__ X, C* __restrict__ Y, size_t rows, int L, int TS, int NF) {
  const size_t total = rows * NF;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % NF);
    const size_t r = idx / NF;
    C out{0, 0};
    if (q <= L - 1) out = X[r * TS + q];
    else if (q >= NF - (L - 1)) out = X[r * TS + (q - NF + TS)];
    Y[idx] = out;
  }
}

// X[r][q] (q < TS) = Y[r][k mod NF] for the frequency k = q (q <= L-1) or q - TS (q >= TS-L+1);
// 0 at the one index of neither range (q = L on MWSS's torus of 2L points).
template <typename C>
__global__ void truncate_kernel(const C* __restrict__ Y, C* __restrict__ X, size_t rows, int L, int TS, int NF) {
  const size_t total = rows * TS;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % TS);
    const size_t r = idx / TS;
    C out{0, 0};
    if (q <= L - 1) out = Y[r * NF + q];
    else if (q >= TS - (L - 1)) out = Y[r * NF + (q - TS + NF)];
    X[idx] = out;
  }
}

template <typename C>
__global__ void weight_fine_kernel(C* __restrict__ Y, size_t rows, int NF, const double* __restrict__ w) {
  using R = typename RealOf<C>::type;
  const size_t total = rows * NF;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const R s = (R)w[idx % NF];
    C v = Y[idx];
    Y[idx] = C{v.x * s, v.y * s};
  }
}

// rows of length TS: row[t] *= nu_t for t < R, row[t] = 0 for t >= R (adjoint of "take the
// rings t < R, times nu").
template <typename C>
__global__ void nu_extend_kernel(C* __restrict__ X, size_t rows, int R, int TS, const double* __restrict__ nu) {
  using Rl = typename RealOf<C>::type;
  const size_t total = rows * TS;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx % TS);
    if (t < R) {
      const Rl s = (Rl)nu[t];
      C v = X[idx];
      X[idx] = C{v.x * s, v.y * s};
    } else {
      X[idx] = C{0, 0};
    }
  }
}

// ring spectra [S][R][W]: X[s][t][k] *= nu_t.
template <typename C>
__global__ void ring_weight_kernel(C* __restrict__ X, size_t S, int R, int W, const double* __restrict__ nu) {
  using Rl = typename RealOf<C>::type;
  const size_t total = S * R * W;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const Rl s = (Rl)nu[(idx / W) % R];
    C v = X[idx];
    X[idx] = C{v.x * s, v.y * s};
  }
}

// Wigner: [b][k'][plane] (k' = n mod K) <-> [b][n+N-1][plane], times a real factor.
template <typename C>
__global__ void gamma_reorder_kernel(const C* __restrict__ in, C* __restrict__ out, int batch, int N,
                                     size_t plane, int to_signal, double scale) {
  using R = typename RealOf<C>::type;
  const int K = 2 * N - 1;
  const size_t total = (size_t)batch * K * plane;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t e = idx % plane;
    const int o = (int)((idx / plane) % K);
    const size_t b = idx / (plane * K);
    int src;
    if (to_signal) {          // output index o = n + N - 1, input index k' = n mod K
      const int n = o - (N - 1);
      src = n >= 0 ? n : n + K;
    } else {                  // output index o = k', input index n + N - 1
      const int n = o <= N - 1 ? o : o - K;
      src = n + N - 1;
    }
    C v = in[(b * K + src) * plane + e];
    out[idx] = C{(R)(v.x * scale), (R)(v.y * scale)};
  }
}

// Real-signal spectra (columns m = 0 .. W-1): X[r][m] *= s for m >= 1; X[r][0] keeps its real
// part only (the m = 0 term of a real signal's spectrum is real).
template <typename C>
__global__ void scale_nonzero_orders_kernel(C* __restrict__ X, size_t rows, int W, double s) {
  using R = typename RealOf<C>::type;
  const size_t total = rows * W;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    C v = X[idx];
    X[idx] = (idx % W == 0) ? C{v.x, (R)0} : C{(R)(v.x * s), (R)(v.y * s)};
  }
}

// out[i] = sum_{p < nparts} parts[p * n + i], in the order of p, for the columns (rows of ld,
// column c0 + m) of the orders |m| in [mlo, mhi).
template <typename C>
__global__ void sum_parts_kernel(const C* __restrict__ parts, C* __restrict__ out, size_t n, int nparts,
                                 int ld, int c0, int mlo, int mhi) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int am = abs((int)(i % ld) - c0);
    if (am < mlo || am >= mhi) continue;
    C acc = parts[i];
    for (int q = 1; q < nparts; ++q) {
      const C v = parts[(size_t)q * n + i];
      acc.x += v.x;
      acc.y += v.y;
    }
    out[i] = acc;
  }
}

}  // namespace

cudaError_t launch_sum_parts(const Plan& p, const void* parts, void* out, int nsig, int nparts,
                             int mlo, int mhi, int ld, int c0, cudaStream_t st) {
  const size_t n = (size_t)nsig * p.nN * p.L * ld;
  if (p.precision == S2GB_FP64)
    sum_parts_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)parts, (double2*)out, n, nparts, ld, c0, mlo, mhi);
  else
    sum_parts_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)parts, (float2*)out, n, nparts, ld, c0, mlo, mhi);
  return launched();
}

static Torus torus_of(const Plan& p) {
  return Torus{p.L, p.R, p.TS, p.sampling == S2GB_MWSS ? 2 * p.L : 2 * p.L - 2};
}

// columns of the phi spectra: P (complex signals) or L (real signals, orders m >= 0)
static int spectra_width(const Plan& p) { return p.real ? p.L : p.P; }

cudaError_t launch_extend(const Plan& p, const void* F, void* G, int nsig, cudaStream_t st) {
  if (!p.TS) return cudaErrorInvalidValue;
  const size_t n = (size_t)nsig * p.MR * p.TS;
  const int mo = p.real ? 0 : p.L - 1;
  const Torus tor = torus_of(p);
  if (p.precision == S2GB_FP64)
    extend_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)F, (double2*)G, nsig, tor, p.nN, p.n_of,
                                                        p.MR, mo, spectra_width(p));
  else
    extend_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)F, (float2*)G, nsig, tor, p.nN, p.n_of,
                                                       p.MR, mo, spectra_width(p));
  return launched();
}

cudaError_t launch_extend_adjoint(const Plan& p, const void* G, void* F, int nsig, cudaStream_t st) {
  if (!p.TS) return cudaErrorInvalidValue;
  const size_t n = (size_t)nsig * p.R * spectra_width(p);
  const int mo = p.real ? 0 : p.L - 1;
  const Torus tor = torus_of(p);
  if (p.precision == S2GB_FP64)
    extend_adjoint_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)G, (double2*)F, nsig, tor, p.nN,
                                                                p.n_of, p.MR, mo, spectra_width(p));
  else
    extend_adjoint_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)G, (float2*)F, nsig, tor, p.nN,
                                                               p.n_of, p.MR, mo, spectra_width(p));
  return launched();
}

cudaError_t launch_scale_nonzero_orders(const Plan& p, void* X, size_t rows, double s, cudaStream_t st) {
  const size_t n = rows * p.L;
  if (p.precision == S2GB_FP64)
    scale_nonzero_orders_kernel<double2><<<grid_for(n), 256, 0, st>>>((double2*)X, rows, p.L, s);
  else
    scale_nonzero_orders_kernel<float2><<<grid_for(n), 256, 0, st>>>((float2*)X, rows, p.L, s);
  return launched();
}

cudaError_t launch_pad(const Plan& p, const void* X, void* Y, int rows, cudaStream_t st) {
  const size_t n = (size_t)rows * p.Nfft;
  if (p.precision == S2GB_FP64)
    pad_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)X, (double2*)Y, (size_t)rows, p.L, p.TS, p.Nfft);
  else
    pad_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)X, (float2*)Y, (size_t)rows, p.L, p.TS, p.Nfft);
  return launched();
}

cudaError_t launch_truncate(const Plan& p, const void* Y, void* X, int rows, cudaStream_t st) {
  const size_t n = (size_t)rows * p.TS;
  if (p.precision == S2GB_FP64)
    truncate_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)Y, (double2*)X, (size_t)rows, p.L, p.TS, p.Nfft);
  else
    truncate_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)Y, (float2*)X, (size_t)rows, p.L, p.TS, p.Nfft);
  return launched();
}

cudaError_t launch_weight_fine(const Plan& p, void* Y, int rows, cudaStream_t st) {
  const size_t n = (size_t)rows * p.Nfft;
  if (p.precision == S2GB_FP64)
    weight_fine_kernel<double2><<<grid_for(n), 256, 0, st>>>((double2*)Y, (size_t)rows, p.Nfft, p.wfine);
  else
    weight_fine_kernel<float2><<<grid_for(n), 256, 0, st>>>((float2*)Y, (size_t)rows, p.Nfft, p.wfine);
  return launched();
}

cudaError_t launch_nu_extend(const Plan& p, void* X, int rows, cudaStream_t st) {
  const size_t n = (size_t)rows * p.TS;
  if (p.precision == S2GB_FP64)
    nu_extend_kernel<double2><<<grid_for(n), 256, 0, st>>>((double2*)X, (size_t)rows, p.R, p.TS, p.nu);
  else
    nu_extend_kernel<float2><<<grid_for(n), 256, 0, st>>>((float2*)X, (size_t)rows, p.R, p.TS, p.nu);
  return launched();
}

cudaError_t launch_ring_weight(const Plan& p, void* X, int nsig, int W, cudaStream_t st) {
  const size_t n = (size_t)nsig * p.R * W;
  if (p.precision == S2GB_FP64)
    ring_weight_kernel<double2><<<grid_for(n), 256, 0, st>>>((double2*)X, (size_t)nsig, p.R, W, p.nu);
  else
    ring_weight_kernel<float2><<<grid_for(n), 256, 0, st>>>((float2*)X, (size_t)nsig, p.R, W, p.nu);
  return launched();
}

cudaError_t zero_nyquist(const Plan& p, void* X, int nsig, cudaStream_t st) {
  if (p.sampling != S2GB_MWSS || p.real) return cudaSuccess;
  const size_t es = p.precision == S2GB_FP64 ? 16 : 8;
  return cudaMemset2DAsync(reinterpret_cast<char*>(X) + (size_t)p.L * es, (size_t)p.P * es, 0, es,
                           (size_t)nsig * p.R, st);
}

cudaError_t launch_gamma_reorder(const Plan& p, const void* in, void* out, int batch, int to_signal,
                                 double scale, cudaStream_t st) {
  const size_t plane = (size_t)p.R * p.P;
  const size_t n = (size_t)batch * p.nN * plane;
  if (p.precision == S2GB_FP64)
    gamma_reorder_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)in, (double2*)out, batch, p.N, plane, to_signal, scale);
  else
    gamma_reorder_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)in, (float2*)out, batch, p.N, plane, to_signal, scale);
  return launched();
}

}  // namespace s2gb
