// Precompute mode of the theta stages (the paper's precompute variant, Sec. 4.4): the Wigner
// d-functions d^l_{m,n}(theta_t) of every (n, m) the theta kernels run are generated once per plan
// by the same recursion as the on-the-fly kernels and kept in device memory; the inverse and
// forward theta stages then read them instead of running the recursion.
//
// Table layout: for each stored (n, m) the rows l = l0 .. L-1 (l0 = max(|m|, |n|)) of L doubles,
// ring index fastest, at tab_off[ni][m + L - 1].  Which (n, m) are stored follows the CTAs of the
// theta kernels: with +-m pairing only n >= 0 (and m >= 0 at n = 0; the partner (-m, -n) reuses the
// table with the sign (-1)^{m-n}), real-signal plans m >= 0, otherwise every (n, m).  A value is
// stored as 0 where the on-the-fly kernels treat the chain as dead (|d| < 2^-kLiveThr), and
// live0[ni][m + L - 1][g] holds the first degree at which one of the 32 rings 32g .. 32g+31 is
// live, so that warps skip the dead prefix of a row (a performance hint only: the stored zeros
// make skipping and not skipping give the same sums).
#include <cuda_runtime.h>

#include <vector>

#include "theta_common.cuh"

namespace s2gb {

namespace {
using namespace theta;

constexpr int kTabChunk = 32;   // degrees of coefficients staged per chunk

// ------------------------------------------------------------------------------------------
// Table construction.  Grid: x = (m + L - 1) * ntiles + tile, y = n index.  Thread tid holds
// KT rings t = tile * KT * 128 + i * 128 + tid.  A tile containing a polar-cap ring runs the
// difference form for all its chains (as the inverse kernel does).
// ------------------------------------------------------------------------------------------
struct TabArgs {
  int L;
  const double* coef;
  const RingData* ring;
  const SeedData* seed;
  double* dtab;
  const size_t* tab_off;
  int* live0;
  int ngroups;
};

template <int KT, bool DIFF>
__device__ __forceinline__ void table_body(const TabArgs& a, int ni, int mi, int tile, size_t off,
                                           double* __restrict__ cs) {
  const int L = a.L, T = 2 * L - 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  const int l0 = sd.l0;
  const double* coef_m = a.coef + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStepN;
  double* rows = a.dtab + off;

  double x[KT], y[KT], v[KT];
  int E[KT], tt[KT], first[KT];
  bool north[KT];
  unsigned nmask[KT];
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    const int t = tile * KT * nt + i * nt + tid;
    tt[i] = t;
    first[i] = L;
    if (t < L) {
      const RingData rd = a.ring[t];
      seed_value(sd, rd, x[i], E[i]);
      v[i] = rd.v;
      north[i] = rd.north;
    } else {
      x[i] = 0.0; E[i] = 1; v[i] = 0.0; north[i] = true;   // inactive: never live
    }
    nmask[i] = north[i] ? 0x80000000u : 0u;
    y[i] = 0.0;
  }

  for (int jc = l0; jc < L; jc += kTabChunk) {
    __syncthreads();
    for (int q = tid; q < kTabChunk * kCoefPerStepN; q += nt) {
      const int j = jc + q / kCoefPerStepN;
      cs[q] = (j < L) ? coef_m[(size_t)jc * kCoefPerStepN + q] : 0.0;
    }
    __syncthreads();
    const int jend = min(kTabChunk, L - jc);
    for (int j8 = 0; j8 < jend; j8 += 8) {
#pragma unroll
      for (int i = 0; i < KT; ++i)
        if (first[i] == L && __any_sync(0xffffffffu, E[i] == 0)) first[i] = jc + j8;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int jj = j8 + u;
        if (jj < jend) {
          const int j = jc + jj;
          // plain chains hold u^j = d^j / gamma_j; the difference form holds d^j itself
          const double fac = DIFF ? 1.0 : cs[jj * kCoefPerStepN + 3];
#pragma unroll
          for (int i = 0; i < KT; ++i)
            if (tt[i] < L) rows[(size_t)(j - l0) * L + tt[i]] = (E[i] == 0) ? x[i] * fac : 0.0;
          if (j < L - 1) {
            const StepN c = stepn_at(cs + jj * kCoefPerStepN);
#pragma unroll
            for (int i = 0; i < KT; ++i) stepn<DIFF>(x[i], y[i], v[i], nmask[i], north[i], c);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < KT; ++i) renorm(x[i], y[i], E[i]);
    }
  }
  const int lane = tid & 31;
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    const int t0 = tt[i] - lane;                     // first ring of this warp's 32
    if (lane == 0 && t0 < L) a.live0[((size_t)ni * T + mi) * a.ngroups + t0 / 32] = first[i];
  }
}

template <int KT>
__global__ void __launch_bounds__(128) dtable_kernel(TabArgs a, int ntiles) {
  __shared__ double cs[kTabChunk * kCoefPerStepN];
  const int L = a.L, T = 2 * L - 1;
  const int mi = blockIdx.x / ntiles, tile = blockIdx.x % ntiles, ni = blockIdx.y;
  const size_t off = a.tab_off[(size_t)ni * T + mi];
  if (off == kNoTable) return;
  const int t_lo = tile * KT * blockDim.x, t_hi = min(L, t_lo + KT * (int)blockDim.x) - 1;
  if (a.ring[t_lo].diff || a.ring[t_hi].diff) table_body<KT, true>(a, ni, mi, tile, off, cs);
  else table_body<KT, false>(a, ni, mi, tile, off, cs);
}

// ------------------------------------------------------------------------------------------
// Inverse theta stage from the table: out[sig][t][m] = sum_l scale_l flm[sig][l][m] d^l_{m,n}(t).
// Grid as the on-the-fly inverse kernel: x = (rank of m) * ntiles + tile, y = n index, z = batch
// group.  Each 8-degree block of a slot's rows is read (coalesced, 8 independent loads per slot)
// unless the whole block is dead for the warp's 32 rings.
// ------------------------------------------------------------------------------------------
template <int KT, int NB, bool PAIR>
__global__ void __launch_bounds__(128) theta_inverse_pre_kernel(InvArgs a, int ntiles) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  __shared__ double2 hs[kTabChunk * NBX];
  const int L = a.L, T = 2 * L - 1;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5;
  const int rank = a.rank0 + (int)(blockIdx.x / ntiles), tile = blockIdx.x % ntiles;
  const int m = a.mpos ? rank : m_of_rank(rank);
  const int ni = PAIR ? (a.nN - 1) / 2 + (int)blockIdx.y : (int)blockIdx.y;
  const int n = ni - (a.nN - 1) / 2;
  if (PAIR && n == 0 && m < 0) return;
  const int mi = m + L - 1;
  const int sig0 = blockIdx.z * NB;
  const int l0 = a.seed[(size_t)ni * T + mi].l0;
  const double* rows = (l0 < L) ? a.dtab + a.tab_off[(size_t)ni * T + mi] : a.dtab;
  const int ngroups = (L + 31) / 32;

  int tt[KT], live[KT];
  double2 acc[KT][NBX];
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    const int t = tile * KT * nt + i * nt + tid;
    const int t0 = tile * KT * nt + i * nt + warp * 32;
    tt[i] = min(t, L - 1);                          // inactive lanes read a valid ring, unused
    live[i] = (t0 < L) ? a.live0[((size_t)ni * T + mi) * ngroups + t0 / 32] : L;
#pragma unroll
    for (int b = 0; b < NBX; ++b) acc[i][b] = make_double2(0.0, 0.0);
  }

  const double* scale = a.scale + (size_t)ni * L;
  for (int jc = l0; jc < L; jc += kTabChunk) {
    __syncthreads();
    for (int q = tid; q < kTabChunk * NBX; q += nt) {
      const int jj = q / NBX, b = q % NBX, j = jc + jj;
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      double2 h = make_double2(0.0, 0.0);
      if (j < L && sl.sig_off >= 0) {
        h = reinterpret_cast<const double2*>(a.flm)[((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0];
        if (a.mpos && m == 0) h.y = 0.0;
        const double s = sl.sign * scale[j];
        h.x *= s; h.y *= s;
      }
      hs[q] = h;
    }
    __syncthreads();
    const int jend = min(kTabChunk, L - jc);
    for (int j8 = 0; j8 < jend; j8 += 8) {
      const int jb = jc + j8;
#pragma unroll
      for (int i = 0; i < KT; ++i) {
        if (jb + 8 <= live[i]) continue;            // dead for all 32 rings of this warp
        double d[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          d[u] = (j8 + u < jend) ? __ldg(rows + (size_t)(jb + u - l0) * L + tt[i]) : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
          for (int b = 0; b < NBX; ++b) {
            const double2 h = hs[(j8 + u) * NBX + b];
            acc[i][b].x = fma(d[u], h.x, acc[i][b].x);
            acc[i][b].y = fma(d[u], h.y, acc[i][b].y);
          }
        }
      }
    }
  }

#pragma unroll
  for (int b = 0; b < NBX; ++b) {
    const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
    if (sl.sig_off < 0) continue;
    const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
#pragma unroll
    for (int i = 0; i < KT; ++i) {
      const int t = tile * KT * nt + i * nt + tid;
      if (t < L) {
        double2* o = reinterpret_cast<double2*>(a.out) + (size_t)sl.sig_off * a.s_sig + t * a.s_t + col * a.s_m;
        *o = acc[i][b];
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Forward theta stage from the table: flm[sig][l][m] = scale_l sum_t d^l_{m,n}(t) g[sig][m][t].
// One CTA per (m, n, batch group) owns all rings, t = i * blockDim + tid; per degree group the
// partial sums are reduced as in the on-the-fly forward kernel (warp reduce-scatter, fixed-order
// cross-warp sum: deterministic).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double reduce_scatter32(double (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int s = 0; s < w; ++s) {
      const double send = up ? v[s] : v[s + w];
      const double keep = up ? v[s + w] : v[s];
      v[s] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}

template <int KT, int NB, bool PAIR>
__global__ void __launch_bounds__(128) theta_forward_pre_kernel(FwdArgs a) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  constexpr int JR = 16 / NBX;
  extern __shared__ double2 smem_pre[];
  const int L = a.L, T = 2 * L - 1;
  const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nt >> 5;
  const int rows = KT * nt;
  double2* gs = smem_pre;                                       // [NBX][rows]
  double* red = reinterpret_cast<double*>(gs + NBX * rows);    // [2][nwarps][32]

  const int m = a.mpos ? a.rank0 + (int)blockIdx.x : m_of_rank(a.rank0 + (int)blockIdx.x);
  const int mi = m + L - 1;
  const int ni = PAIR ? (a.nN - 1) / 2 + (int)blockIdx.y : (int)blockIdx.y;
  const int n = ni - (a.nN - 1) / 2;
  if (PAIR && n == 0 && m < 0) return;
  const int sig0 = blockIdx.z * NB;
  const int l0 = a.seed[(size_t)ni * T + mi].l0;
  const double* scale = a.scale + (size_t)ni * L;
  const int ngroups = (L + 31) / 32;

  const int lz = min(l0, L);
  for (int q = tid; q < NBX * lz; q += nt) {
    const int b = q / lz, j = q % lz;
    const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
    if (sl.sig_off >= 0)
      reinterpret_cast<double2*>(a.flm)[((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0] =
          make_double2(0.0, 0.0);
  }
  if (l0 >= L) return;
  const double* trows = a.dtab + a.tab_off[(size_t)ni * T + mi];

  for (int q = tid; q < NBX * rows; q += nt) {
    const int b = q / rows, t = q % rows;
    const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
    double2 g = make_double2(0.0, 0.0);
    if (t < L && sl.sig_off >= 0) {
      const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
      g = reinterpret_cast<const double2*>(a.g)[(size_t)sl.sig_off * a.s_sig + t * a.s_t + col * a.s_m];
      const double w = (a.use_nu ? a.nu[t] : 1.0) * sl.sign;
      g.x *= w; g.y *= w;
    }
    gs[q] = g;
  }
  __syncthreads();

  int tt[KT], live[KT];
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    const int t0 = i * nt + warp * 32;
    tt[i] = min(i * nt + tid, L - 1);               // inactive lanes read a valid ring; g is 0 there
    live[i] = (t0 < L) ? a.live0[((size_t)ni * T + mi) * ngroups + t0 / 32] : L;
  }

  int buf = 0;
  for (int j0 = l0; j0 < L; j0 += JR) {
    double p[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) p[s] = 0.0;
#pragma unroll
    for (int i = 0; i < KT; ++i) {
      if (j0 + JR <= live[i]) continue;              // dead for the warp's 32 rings
      double d[JR];
#pragma unroll
      for (int jr = 0; jr < JR; ++jr)
        d[jr] = (j0 + jr < L) ? __ldg(trows + (size_t)(j0 + jr - l0) * L + tt[i]) : 0.0;
      const int pos = i * nt + tid;
#pragma unroll
      for (int b = 0; b < NBX; ++b) {
        const double2 g = gs[b * rows + pos];
#pragma unroll
        for (int jr = 0; jr < JR; ++jr) {
          p[jr * 2 * NBX + 2 * b] = fma(d[jr], g.x, p[jr * 2 * NBX + 2 * b]);
          p[jr * 2 * NBX + 2 * b + 1] = fma(d[jr], g.y, p[jr * 2 * NBX + 2 * b + 1]);
        }
      }
    }
    const double s = reduce_scatter32(p);
    red[(buf * nwarps + warp) * 32 + lane] = s;
    __syncthreads();
    if (warp == 0) {
      double tot = red[(buf * nwarps) * 32 + lane];
      for (int w = 1; w < nwarps; ++w) tot += red[(buf * nwarps + w) * 32 + lane];
      const int jr = lane / (2 * NBX), b = (lane / 2) % NBX, reim = lane & 1;
      const int j = j0 + jr;
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      if (j < L && sl.sig_off >= 0) {
        double* o = reinterpret_cast<double*>(reinterpret_cast<double2*>(a.flm) +
                                              ((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0);
        o[reim] = tot * scale[j];
      }
    }
    buf ^= 1;
  }
}

template <int KT, int NB, bool PAIR>
cudaError_t launch_inv_pre(const Plan& p, const InvArgs& a, cudaStream_t st) {
  const int nt = 128;
  const int ntiles = (p.L + KT * nt - 1) / (KT * nt);
  dim3 grid(a.nrank * ntiles, PAIR ? (a.nN + 1) / 2 : a.nN, (a.nsig + NB - 1) / NB);
  theta_inverse_pre_kernel<KT, NB, PAIR><<<grid, nt, 0, st>>>(a, ntiles);
  return launched();
}

template <int NB, bool PAIR>
cudaError_t launch_inv_pre_nb(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (p.L <= 128) return launch_inv_pre<1, NB, PAIR>(p, a, st);
  if (p.L <= 512) return launch_inv_pre<2, NB, PAIR>(p, a, st);
  return launch_inv_pre<4, NB, PAIR>(p, a, st);
}

template <int KT, int NB, bool PAIR>
cudaError_t launch_fwd_pre(const Plan& p, const FwdArgs& a, int nt, cudaStream_t st) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  const int rows = KT * nt;
  const size_t smem = sizeof(double2) * NBX * rows + sizeof(double) * 2 * (nt / 32) * 32;
  auto kern = theta_forward_pre_kernel<KT, NB, PAIR>;
  cudaError_t e = set_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nrank, PAIR ? (a.nN + 1) / 2 : a.nN, (a.nsig + NB - 1) / NB);
  kern<<<grid, nt, smem, st>>>(a);
  return launched();
}

// rows = KT * nt >= L with nt a multiple of 32 (<= 128)
template <int NB, bool PAIR>
cudaError_t launch_fwd_pre_nb(const Plan& p, const FwdArgs& a, cudaStream_t st) {
  const int L = p.L;
  auto nt_for = [L](int kt) { return ((L + kt - 1) / kt + 31) / 32 * 32; };
  if (L <= 128) return launch_fwd_pre<1, NB, PAIR>(p, a, nt_for(1), st);
  if (L <= 256) return launch_fwd_pre<2, NB, PAIR>(p, a, nt_for(2), st);
  if (L <= 512) return launch_fwd_pre<4, NB, PAIR>(p, a, nt_for(4), st);
  if (L <= 1024) return launch_fwd_pre<8, NB, PAIR>(p, a, nt_for(8), st);
  return launch_fwd_pre<16, NB, PAIR>(p, a, nt_for(16), st);
}

}  // namespace

int build_dtable(Plan* p, size_t* bytes) {
  const int L = p->L, T = p->T, nN = p->nN;
  std::vector<int> n_of(nN);
  if (cudaMemcpy(n_of.data(), p->n_of, sizeof(int) * nN, cudaMemcpyDeviceToHost) != cudaSuccess)
    return S2GB_ECUDA;
  const bool pair = paired_plan(*p);
  std::vector<size_t> off((size_t)nN * T, kNoTable);
  size_t total = 0;
  for (int ni = 0; ni < nN; ++ni) {
    const int n = n_of[ni], an = n < 0 ? -n : n;
    for (int mi = 0; mi < T; ++mi) {
      const int m = mi - (L - 1), am = m < 0 ? -m : m;
      bool stored;
      if (p->real) stored = m >= 0;
      else if (pair) stored = n > 0 || (n == 0 && m >= 0);
      else stored = true;
      const int l0 = am > an ? am : an;
      if (!stored || l0 >= L) continue;
      off[(size_t)ni * T + mi] = total;
      total += (size_t)(L - l0) * L;
    }
  }
  const int ngroups = (L + 31) / 32;
  if (cudaMalloc((void**)&p->dtab, total * sizeof(double) + 64) != cudaSuccess) return S2GB_ENOMEM;
  if (cudaMalloc((void**)&p->tab_off, off.size() * sizeof(size_t)) != cudaSuccess) return S2GB_ENOMEM;
  if (cudaMalloc((void**)&p->live0, (size_t)nN * T * ngroups * sizeof(int)) != cudaSuccess) return S2GB_ENOMEM;
  *bytes += total * sizeof(double) + off.size() * sizeof(size_t) + (size_t)nN * T * ngroups * sizeof(int);
  if (cudaMemcpy(p->tab_off, off.data(), off.size() * sizeof(size_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return S2GB_ECUDA;
  if (cudaMemset(p->live0, 0, (size_t)nN * T * ngroups * sizeof(int)) != cudaSuccess) return S2GB_ECUDA;
  TabArgs a{L, p->coef, p->ring, p->seed, p->dtab, p->tab_off, p->live0, ngroups};
  constexpr int KT = 4;
  const int ntiles = (L + KT * 128 - 1) / (KT * 128);
  dtable_kernel<KT><<<dim3(T * ntiles, nN), 128>>>(a, ntiles);
  if (launched() != cudaSuccess) return S2GB_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return S2GB_ECUDA;
  return S2GB_OK;
}

cudaError_t launch_theta_inverse_pre(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (paired_plan(p)) {
    if (a.nsig >= 2) return launch_inv_pre_nb<2, true>(p, a, st);
    return launch_inv_pre_nb<1, true>(p, a, st);
  }
  if (a.nsig >= 4) return launch_inv_pre_nb<4, false>(p, a, st);
  if (a.nsig >= 2) return launch_inv_pre_nb<2, false>(p, a, st);
  return launch_inv_pre_nb<1, false>(p, a, st);
}

// Staged ring data NBX * rows * 16 bytes stays <= 64 KB (3 CTAs per SM): above L = 1024 one signal
// per CTA.
cudaError_t launch_theta_forward_pre(const Plan& p, const FwdArgs& a, cudaStream_t st) {
  const bool big = p.L > 1024;
  if (paired_plan(p)) {
    if (a.nsig >= 2 && !big) return launch_fwd_pre_nb<2, true>(p, a, st);
    return launch_fwd_pre_nb<1, true>(p, a, st);
  }
  if (a.nsig >= 4 && !big) return launch_fwd_pre_nb<4, false>(p, a, st);
  if (a.nsig >= 2) return launch_fwd_pre_nb<2, false>(p, a, st);
  return launch_fwd_pre_nb<1, false>(p, a, st);
}

}  // namespace s2gb
