// Memory-bound glue between the FFT stages of the MW transforms: the theta torus extension of
// Sec. 4.2.2 and its adjoint, Fourier-domain zero padding and truncation, the fine-grid weights
// of the forward quadrature, and the gamma-axis reordering of the Wigner transform.
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

// G[s][r][t'] (t' < T) from F[s][t][k]:  t' < L-1: F[t'];  t' = L-1: (1+sigma)/2 F[L-1];
// t' >= L: sigma F[2L-2-t'];  sigma = (-1)^{m-n}.  Row r of G is order m = r - mo (MR rows); F has
// rows of FW columns with column k = m mod T (complex signals: MR = FW = T, mo = L-1; real
// signals, m >= 0 only: MR = FW = L, mo = 0).
template <typename C>
__global__ void extend_kernel(const C* __restrict__ F, C* __restrict__ G, int S, int L, int nN,
                              const int* __restrict__ n_of, int MR, int mo, int FW) {
  const int T = 2 * L - 1;
  const size_t total = (size_t)S * MR * T;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int tp = (int)(idx % T);
    const int r = (int)((idx / T) % MR);
    const int s = (int)(idx / ((size_t)T * MR));
    const int m = r - mo;
    const int k = m >= 0 ? m : m + T;
    const int n = n_of[s % nN];
    const bool odd = ((m - n) & 1) != 0;
    C out;
    if (tp < L - 1) {
      out = F[((size_t)s * L + tp) * FW + k];
    } else if (tp == L - 1) {
      out = odd ? C{0, 0} : F[((size_t)s * L + tp) * FW + k];
    } else {
      C v = F[((size_t)s * L + (2 * L - 2 - tp)) * FW + k];
      out = odd ? C{-v.x, -v.y} : v;
    }
    G[idx] = out;
  }
}

// Adjoint of extend_kernel: F[s][t][k] = G[s][r][t] + sigma G[s][r][2L-2-t] (t < L-1),
// F[s][L-1][k] = (1+sigma)/2 G[s][r][L-1], for every column k of F (FW = MR columns).
template <typename C>
__global__ void extend_adjoint_kernel(const C* __restrict__ G, C* __restrict__ F, int S, int L, int nN,
                                      const int* __restrict__ n_of, int MR, int mo) {
  const int T = 2 * L - 1;
  const size_t total = (size_t)S * L * MR;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % MR);
    const int t = (int)((idx / MR) % L);
    const int s = (int)(idx / ((size_t)MR * L));
    const int m = k <= L - 1 ? k : k - T;
    const int r = m + mo;
    const int n = n_of[s % nN];
    const bool odd = ((m - n) & 1) != 0;
    const C* row = G + ((size_t)s * MR + r) * T;
    C out;
    if (t < L - 1) {
      C a = row[t], b = row[2 * L - 2 - t];
      out = odd ? C{a.x - b.x, a.y - b.y} : C{a.x + b.x, a.y + b.y};
    } else {
      out = odd ? C{0, 0} : row[t];
    }
    F[idx] = out;
  }
}

// Y[r][q] (q < NF) = X[r][k mod T] for the frequency k = q (q <= L-1) or q - NF (q >= NF-L+1).
template <typename C>
__global__ void pad_kernel(const C* __restrict__ X, C* __restrict__ Y, size_t rows, int L, int NF) {
  const int T = 2 * L - 1;
  const size_t total = rows * NF;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % NF);
    const size_t r = idx / NF;
    C out{0, 0};
    if (q <= L - 1) out = X[r * T + q];
    else if (q >= NF - (L - 1)) out = X[r * T + (q - NF + T)];
    Y[idx] = out;
  }
}

// X[r][q] (q < T) = Y[r][k mod NF] for the frequency k = q (q <= L-1) or q - T (q >= L).
template <typename C>
__global__ void truncate_kernel(const C* __restrict__ Y, C* __restrict__ X, size_t rows, int L, int NF) {
  const int T = 2 * L - 1;
  const size_t total = rows * T;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % T);
    const size_t r = idx / T;
    X[idx] = (q <= L - 1) ? Y[r * NF + q] : Y[r * NF + (q - T + NF)];
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

// rows of length T: row[t] *= nu_t for t < L, row[t] = 0 for t >= L (adjoint of "take t < L, * nu").
template <typename C>
__global__ void nu_extend_kernel(C* __restrict__ X, size_t rows, int L, const double* __restrict__ nu) {
  using R = typename RealOf<C>::type;
  const int T = 2 * L - 1;
  const size_t total = rows * T;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx % T);
    if (t < L) {
      const R s = (R)nu[t];
      C v = X[idx];
      X[idx] = C{v.x * s, v.y * s};
    } else {
      X[idx] = C{0, 0};
    }
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

cudaError_t launch_extend(const Plan& p, const void* F, void* G, int nsig, cudaStream_t st) {
  const size_t n = (size_t)nsig * p.MR * p.T;
  const int mo = p.real ? 0 : p.L - 1;
  if (p.precision == S2GB_FP64)
    extend_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)F, (double2*)G, nsig, p.L, p.nN, p.n_of,
                                                        p.MR, mo, p.MR);
  else
    extend_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)F, (float2*)G, nsig, p.L, p.nN, p.n_of,
                                                       p.MR, mo, p.MR);
  return launched();
}

cudaError_t launch_extend_adjoint(const Plan& p, const void* G, void* F, int nsig, cudaStream_t st) {
  const size_t n = (size_t)nsig * p.L * p.MR;
  const int mo = p.real ? 0 : p.L - 1;
  if (p.precision == S2GB_FP64)
    extend_adjoint_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)G, (double2*)F, nsig, p.L, p.nN,
                                                                p.n_of, p.MR, mo);
  else
    extend_adjoint_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)G, (float2*)F, nsig, p.L, p.nN,
                                                               p.n_of, p.MR, mo);
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
    pad_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)X, (double2*)Y, (size_t)rows, p.L, p.Nfft);
  else
    pad_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)X, (float2*)Y, (size_t)rows, p.L, p.Nfft);
  return launched();
}

cudaError_t launch_truncate(const Plan& p, const void* Y, void* X, int rows, cudaStream_t st) {
  const size_t n = (size_t)rows * p.T;
  if (p.precision == S2GB_FP64)
    truncate_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)Y, (double2*)X, (size_t)rows, p.L, p.Nfft);
  else
    truncate_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)Y, (float2*)X, (size_t)rows, p.L, p.Nfft);
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
  const size_t n = (size_t)rows * p.T;
  if (p.precision == S2GB_FP64)
    nu_extend_kernel<double2><<<grid_for(n), 256, 0, st>>>((double2*)X, (size_t)rows, p.L, p.nu);
  else
    nu_extend_kernel<float2><<<grid_for(n), 256, 0, st>>>((float2*)X, (size_t)rows, p.L, p.nu);
  return launched();
}

cudaError_t launch_gamma_reorder(const Plan& p, const void* in, void* out, int batch, int to_signal,
                                 double scale, cudaStream_t st) {
  const size_t plane = (size_t)p.L * p.T;
  const size_t n = (size_t)batch * p.nN * plane;
  if (p.precision == S2GB_FP64)
    gamma_reorder_kernel<double2><<<grid_for(n), 256, 0, st>>>((const double2*)in, (double2*)out, batch, p.N, plane, to_signal, scale);
  else
    gamma_reorder_kernel<float2><<<grid_for(n), 256, 0, st>>>((const float2*)in, (float2*)out, batch, p.N, plane, to_signal, scale);
  return launched();
}

}  // namespace s2gb
