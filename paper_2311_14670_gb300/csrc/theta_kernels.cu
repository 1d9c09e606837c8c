// Theta stages of the spin-s SHT (Sec. 4.1, Eqs. disc_ish_expanded and disc_sh_expanded) with the
// Wigner d-functions generated on the fly and interleaved with the contraction (Sec. 4.4).
//
// Recursion.  For fixed (m, n, theta) the functions d^j_{mn}(theta) obey, for j >= l0 =
// max(|m|,|n|) and with d^{l0-1} = 0, the three-term recurrence in the degree
//     d^{j+1} = A_j (cos theta - B_j) d^j - C_j d^{j-1}
// (coefficients in plan.cu).  Each thread owns KT (m, theta) chains; the state lives in registers.
// Ascending j the wanted solution dominates, so the recurrence is stable.  It is run in the
// half-angle variable v = 2 sin^2(theta/2) (north rings) or v = 2 cos^2(theta/2) (south rings),
//     P_j = A_j (cos theta - B_j) = K_n - A_j v   or   K_s + A_j v,
// because cos theta itself cannot resolve theta near the poles (an error of one ulp in cos theta
// shifts d^l by ~l^2 ulp there).  On rings with sin(theta) < kPoleSin the recurrence is nearly
// degenerate (its characteristic roots approach +-1) and amplifies rounding of the state by
// ~1/sin(theta); there the "difference form" carries e^j = d^j - sigma d^{j-1} (sigma = +1 north,
// -1 south):
//     e^{j+1} = (P_j - sigma (1 + C_j)) d^j + sigma C_j e^j,    d^{j+1} = sigma d^j + e^{j+1},
// whose coefficient P_j - sigma(1+C_j) = Kd - (+-A_j v) is small and precomputed accurately.
// Both forms are carried normalised along the whole chain (u^j = d^j / gamma_j plain, e^j / eta_j
// in the difference form; products of the C_k, plan.cu), which leaves 2 FMA per plain step and
// 3 per difference step; gamma_j goes into the contraction's coefficient or output scale.
//
// Range.  Starting values d^{l0} (Eq. "initial_values" via the symmetries of Sec. 3.3) can be as
// small as 2^-20000.  A chain keeps its value as x * 2^-E with an integer E >= 0.  While E > 0 the
// chain is "dead": its true magnitude is below 2^-kLiveThr and it contributes nothing (exactly as
// in float64, where such products vanish against the O(1) sum).  Every few steps the exponent of x
// is inspected on the integer pipe: a chain whose true magnitude has grown past 2^-kLiveThr is
// converted to unscaled form (E = 0) and contributes from then on; a dead chain whose x grew past
// 2^kRescale is rescaled by an exact power of two.  Once unscaled, |d| <= 1 and never underflows
// (ascending l leaves the forbidden region for good), so no further checks are needed.  This is
// the running renormalisation of Sec. 3.4 in exact power-of-two form.
#include <cuda_runtime.h>

#include "theta_common.cuh"

namespace s2gb {

namespace {
using namespace theta;

// ------------------------------------------------------------------------------------------
// Inverse theta stage: out[sig][t][m] = sum_{l >= l0} scale_l flm[sig][l][m] d^l_{m,n}(theta_t).
// Grid: x = (rank of m) * ntiles + tile, y = n index, z = batch group of NB signals.
// Each thread owns KT rings t = tile*KT*blockDim + i*blockDim + threadIdx.x.  The coefficients
// flm[.][l][m] * scale_l for a chunk of kChunk degrees are staged in shared memory.
// ------------------------------------------------------------------------------------------
constexpr int kChunk = 32;

template <int KT, int NB, bool DIFF, bool PAIR>
__device__ __forceinline__ void inverse_body(const InvArgs& a, int m, int ni, int n, int tile, int l0,
                                             double2* __restrict__ hs, double* __restrict__ cs) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  const int L = a.L, T = 2 * L - 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mi = m + L - 1;
  const int sig0 = blockIdx.z * NB;
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  const double* coef_m = a.coef + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStepN;

  double x[KT], y[KT], v[KT];
  int E[KT], tt[KT];
  bool north[KT];
  unsigned nmask[KT];
  double2 acc[KT][NBX];
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    const int t = a.ring0 + tile * KT * nt + i * nt + tid;
    tt[i] = t;
    if (t < a.nring) {
      const RingData rd = a.ring[t];
      seed_value(sd, rd, x[i], E[i]);
      v[i] = rd.v;
      north[i] = rd.north;
    } else {
      x[i] = 0.0; E[i] = 0; v[i] = 0.0; north[i] = true;
    }
    nmask[i] = north[i] ? 0x80000000u : 0u;
    y[i] = 0.0;   // plain: u^{l0-1} = d^{l0-1} = 0; difference form: ehat^{l0} = 0 (its weight C_{l0} is 0)
#pragma unroll
    for (int b = 0; b < NBX; ++b) acc[i][b] = make_double2(0.0, 0.0);
  }

  const double* scale = a.scale + (size_t)ni * L;   // the same for n and -n
  for (int jc = l0; jc < L; jc += kChunk) {
    __syncthreads();
    for (int q = tid; q < kChunk * NBX; q += nt) {
      const int jj = q / NBX, b = q % NBX, j = jc + jj;
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      double2 h = make_double2(0.0, 0.0);
      if (j < L && sl.sig_off >= 0) {
        h = reinterpret_cast<const double2*>(a.flm)[((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0];
        if (a.mpos && m == 0) h.y = 0.0;      // real signals: flm(l, 0) is real
        // plain chains carry u^j = d^j / gamma_j: fold gamma_j into the coefficient
        const double s = sl.sign * (DIFF ? scale[j] : scale[j] * coef_m[(size_t)j * kCoefPerStepN + 3]);
        h.x *= s; h.y *= s;
      }
      hs[q] = h;
    }
    for (int q = tid; q < kChunk * kCoefPerStepN; q += nt) {
      const int j = jc + q / kCoefPerStepN;
      cs[q] = (j < L) ? coef_m[(size_t)jc * kCoefPerStepN + q] : 0.0;
    }
    __syncthreads();
    const int jend = min(kChunk, L - jc);
    for (int j8 = 0; j8 < jend; j8 += 8) {
      // chains that are dead in every lane of the warp skip their contraction (warp-uniform)
      unsigned live = 0;
#pragma unroll
      for (int i = 0; i < KT; ++i) live |= (__any_sync(0xffffffffu, E[i] == 0) ? 1u : 0u) << i;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int jj = j8 + u;
        if (jj < jend) {
          double2 h[NBX];
#pragma unroll
          for (int b = 0; b < NBX; ++b) h[b] = hs[jj * NBX + b];
#pragma unroll
          for (int i = 0; i < KT; ++i) {
            if ((live >> i) & 1u) {
              const double xl = (E[i] == 0) ? x[i] : 0.0;
#pragma unroll
              for (int b = 0; b < NBX; ++b) {
                acc[i][b].x = fma(xl, h[b].x, acc[i][b].x);
                acc[i][b].y = fma(xl, h[b].y, acc[i][b].y);
              }
            }
          }
          if (jc + jj < L - 1) {
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

#pragma unroll
  for (int b = 0; b < NBX; ++b) {
    const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
    if (sl.sig_off < 0) continue;
    const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
#pragma unroll
    for (int i = 0; i < KT; ++i) {
      if (tt[i] < a.nring) {
        double2* o = reinterpret_cast<double2*>(a.out) + (size_t)sl.sig_off * a.s_sig + tt[i] * a.s_t + col * a.s_m;
        *o = acc[i][b];
      }
    }
  }
}

// Grid: x = (rank of m) * ntiles + tile, y = n index (with pairing: only n >= 0, and for n = 0 only
// m >= 0 -- the CTA of (m, n) also produces (-m, -n)), z = batch group of NB signals.
template <int KT, int NB, bool PAIR>
__global__ void __launch_bounds__(128) theta_inverse_kernel(InvArgs a, int ntiles) {
  __shared__ double2 hs[kChunk * (PAIR ? 2 * NB : NB)];
  __shared__ double cs[kChunk * kCoefPerStepN];
  const int L = a.L;
  const int rank = a.rank0 + (int)(blockIdx.x / ntiles), tile = blockIdx.x % ntiles;
  const int m = a.mpos ? rank : m_of_rank(rank);
  const int ni = PAIR ? (a.nN - 1) / 2 + (int)blockIdx.y : (int)blockIdx.y;
  const int n = ni - (a.nN - 1) / 2;          // used only with pairing (n-set symmetric about 0)
  if (PAIR && n == 0 && m < 0) return;        // produced by the CTA of -m
  const int l0 = a.seed[(size_t)ni * (2 * L - 1) + m + L - 1].l0;   // max(|m|, |n|)
  // Does this tile contain a ring that needs the difference form?
  const int t_lo = a.ring0 + tile * KT * blockDim.x, t_hi = min(a.nring, t_lo + KT * (int)blockDim.x) - 1;
  const bool diff = a.ring[t_lo].diff || a.ring[t_hi].diff;
  if (diff) inverse_body<KT, NB, true, PAIR>(a, m, ni, n, tile, l0, hs, cs);
  else inverse_body<KT, NB, false, PAIR>(a, m, ni, n, tile, l0, hs, cs);
}

// ------------------------------------------------------------------------------------------
// Forward theta stage: flm[sig][l][m] = scale_l sum_t d^l_{m,n}(theta_t) g[sig][m][t] (* nu_t).
// One CTA per (m, n, batch group) owns all rings of the launch: thread tid holds rings
// t = row0 + i*blockDim + tid (the last slot the last blockDim rings).
// Per degree every thread forms partial sums over its KT rings (FMA chains); partial sums of
// JR = 16/NB consecutive degrees (32 doubles) are reduced across the warp by a reduce-scatter
// (31 additions per lane for 32 values, lane l ends with value l), then across warps through
// shared memory in a fixed order: the result is deterministic.
// The difference form is used on the first and the last ring slot, which hold the polar caps
// (sin theta < kPoleSin covers fewer than L/20 rings at either end, and a slot holds >= L/16), or
// on all slots when PAT == 1.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_reduce_scatter32(double (&v)[32]) {
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

template <int KT, int NB, int PAT, bool PAIR>
__global__ void __launch_bounds__(128) theta_forward_kernel(FwdArgs a) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  constexpr int JR = 16 / NBX;           // degrees per reduction group
  extern __shared__ double2 smem[];
  const int L = a.L, T = 2 * L - 1;
  const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nt >> 5;
  const int rows = KT * nt;                // padded ring count
  const int R = a.nrows, r0 = a.row0;      // this launch's rings: [r0, r0 + R)
  double2* const outb = a.part ? reinterpret_cast<double2*>(a.part) + a.part_off
                               : reinterpret_cast<double2*>(a.flm);
  double2* gs = smem;                                          // [NBX][rows]
  double* red = reinterpret_cast<double*>(gs + NBX * rows);   // [2][nwarps][32]
  double* vs = red + 2 * nwarps * 32;                          // [rows]

  const int m = a.mpos ? a.rank0 + (int)blockIdx.x : m_of_rank(a.rank0 + (int)blockIdx.x);
  const int mi = m + L - 1;
  const int ni = PAIR ? (a.nN - 1) / 2 + (int)blockIdx.y : (int)blockIdx.y;
  const int n = ni - (a.nN - 1) / 2;          // used only with pairing
  if (PAIR && n == 0 && m < 0) return;        // produced by the CTA of -m
  const int sig0 = blockIdx.z * NB;
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  const int l0 = sd.l0;
  const double* scale = a.scale + (size_t)ni * L;   // the same for n and -n

  // zero the degrees l < l0 of the CTA's columns
  const int lz = min(l0, L);
  for (int q = tid; q < NBX * lz; q += nt) {
    const int b = q / lz, j = q % lz;
    const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
    if (sl.sig_off >= 0) outb[((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0] = make_double2(0.0, 0.0);
  }
  if (l0 >= L) return;

  // stage g (times the ring fold factors and the pairing sign) and the ring variables
  for (int q = tid; q < NBX * rows; q += nt) {
    const int b = q / rows, pos = q % rows;
    const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
    bool act;
    const int t = r0 + ring_of<KT>(pos / nt, pos % nt, nt, R, act);
    double2 g = make_double2(0.0, 0.0);
    if (act && sl.sig_off >= 0) {
      const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
      g = reinterpret_cast<const double2*>(a.g)[(size_t)sl.sig_off * a.s_sig + t * a.s_t + col * a.s_m];
      const double w = (a.use_nu ? a.nu[t] : 1.0) * sl.sign;
      g.x *= w; g.y *= w;
    }
    gs[q] = g;
  }
  for (int pos = tid; pos < rows; pos += nt) {
    bool act;
    const int t = r0 + ring_of<KT>(pos / nt, pos % nt, nt, R, act);
    vs[pos] = act ? a.ring[t].v : 0.0;
  }
  __syncthreads();

  double x[KT], y[KT];
  int E[KT];
  bool north[KT];
  unsigned nmask[KT];
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    bool act;
    const int t = r0 + ring_of<KT>(i, tid, nt, R, act);
    if (act) {
      const RingData rd = a.ring[t];
      seed_value(sd, rd, x[i], E[i]);
      north[i] = rd.north;
    } else {
      x[i] = 0.0; E[i] = 0; north[i] = true;
    }
    nmask[i] = north[i] ? 0x80000000u : 0u;
    y[i] = 0.0;   // plain: u^{l0-1} = 0; difference form: ehat^{l0} = 0 (weight C_{l0} = 0)
  }

  const double* coef_m = a.coef + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStepN;
  int buf = 0;
  for (int j0 = l0; j0 < L; j0 += JR) {
    double p[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) p[s] = 0.0;
    // chains that are dead in every lane of the warp skip their contraction (warp-uniform)
    unsigned live = 0;
#pragma unroll
    for (int i = 0; i < KT; ++i) live |= (__any_sync(0xffffffffu, E[i] == 0) ? 1u : 0u) << i;
#pragma unroll
    for (int jr = 0; jr < JR; ++jr) {
      const int j = j0 + jr;
      if (j < L) {
        const double2* c2 = reinterpret_cast<const double2*>(coef_m + (size_t)j * kCoefPerStepN);
        const double2 c01 = __ldg(c2), c23 = __ldg(c2 + 1), c45 = __ldg(c2 + 2), c67 = __ldg(c2 + 3),
                      c89 = __ldg(c2 + 4);
        const StepN c = {c01.x, c01.y, c23.x, c23.y, c45.x, c45.y, c67.x, c67.y, c89.x, c89.y};
#pragma unroll
        for (int i = 0; i < KT; ++i) {
          if ((live >> i) & 1u) {
            // partial sums are kept in units of u^j = d^j / gamma_j (rescaled at the output)
            const bool dslot = (PAT == 1) || (PAT == 0 && (i == 0 || i == KT - 1));
            double xl = (E[i] == 0) ? x[i] : 0.0;
            if (dslot) xl *= c.ig;
            const int pos = i * nt + tid;
#pragma unroll
            for (int b = 0; b < NBX; ++b) {
              const double2 g = gs[b * rows + pos];
              p[jr * 2 * NBX + 2 * b] = fma(xl, g.x, p[jr * 2 * NBX + 2 * b]);
              p[jr * 2 * NBX + 2 * b + 1] = fma(xl, g.y, p[jr * 2 * NBX + 2 * b + 1]);
            }
          }
        }
        if (j < L - 1) {
#pragma unroll
          for (int i = 0; i < KT; ++i) {
            const double v = vs[i * nt + tid];
            const bool dslot = (PAT == 1) || (PAT == 0 && (i == 0 || i == KT - 1));
            if (dslot) stepn<true>(x[i], y[i], v, nmask[i], north[i], c);
            else stepn<false>(x[i], y[i], v, nmask[i], north[i], c);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < KT; ++i) renorm(x[i], y[i], E[i]);

    // reduce the 32 partial sums of this group
    const double s = warp_reduce_scatter32(p);
    red[(buf * nwarps + warp) * 32 + lane] = s;
    __syncthreads();
    if (warp == 0) {
      double tot = red[(buf * nwarps) * 32 + lane];
      for (int w = 1; w < nwarps; ++w) tot += red[(buf * nwarps + w) * 32 + lane];
      const int jr = lane / (2 * NBX), b = (lane / 2) % NBX, reim = lane & 1;
      const int j = j0 + jr;
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      if (j < L && sl.sig_off >= 0) {
        double* o = reinterpret_cast<double*>(outb + ((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0);
        o[reim] = tot * (scale[j] * coef_m[(size_t)j * kCoefPerStepN + 3]);   // * gamma_j
      }
    }
    buf ^= 1;
  }
}

template <int KT, int NB, bool PAIR>
cudaError_t launch_inv(const Plan& p, const InvArgs& a, cudaStream_t st) {
  const int nt = 128;
  const int ntiles = (a.nring - a.ring0 + KT * nt - 1) / (KT * nt);
  if (ntiles == 0) return cudaSuccess;          // no rings for the recursion (MWSS, L = 1)
  dim3 grid(a.nrank * ntiles, PAIR ? (a.nN + 1) / 2 : a.nN, (a.nsig + NB - 1) / NB);
  theta_inverse_kernel<KT, NB, PAIR><<<grid, nt, 0, st>>>(a, ntiles);
  return launched();
}

template <int NB, bool PAIR>
cudaError_t launch_inv_nb(const Plan& p, const InvArgs& a, cudaStream_t st) {
  const int rings = a.nring - a.ring0;
  if (rings <= 128) return launch_inv<1, NB, PAIR>(p, a, st);
  if (rings <= 512) return launch_inv<2, NB, PAIR>(p, a, st);
  return launch_inv<4, NB, PAIR>(p, a, st);
}

template <int KT, int NB, int PAT, bool PAIR>
cudaError_t launch_fwd(const Plan& p, const FwdArgs& a, int nt, cudaStream_t st) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  const int rows = KT * nt;
  const size_t smem = sizeof(double2) * NBX * rows + sizeof(double) * (2 * (nt / 32) * 32 + rows);
  auto kern = theta_forward_kernel<KT, NB, PAT, PAIR>;
  cudaError_t e = set_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nrank, PAIR ? (a.nN + 1) / 2 : a.nN, (a.nsig + NB - 1) / NB);
  kern<<<grid, nt, smem, st>>>(a);
  return launched();
}

template <int NB, bool PAIR>
cudaError_t launch_fwd_nb(const Plan& p, const FwdArgs& a0, cudaStream_t st) {
  const int R = p.nint;    // rings of the recursion kernels: [ring0, ring0 + nint)
  FwdArgs a = a0;
  a.row0 = p.ring0;
  a.nrows = R;
  a.part = nullptr;
  a.part_off = 0;
  if (R <= 128) return launch_fwd<1, NB, 1, PAIR>(p, a, R > 32 ? ((R + 31) / 32) * 32 : 32, st);
  if (R <= 256) return launch_fwd<2, NB, 1, PAIR>(p, a, 128, st);
  if (R <= 512) return launch_fwd<4, NB, 0, PAIR>(p, a, 128, st);
  // Unpaired: 16 rings per thread (64 threads) halve the cross-thread reduction; paired CTAs carry
  // twice the signal slots and run better with 8 rings per thread (measured on GB300).
  if (R <= 1024) {
    if (PAIR) return launch_fwd<8, NB, 0, PAIR>(p, a, 128, st);
    return launch_fwd<16, NB, 0, PAIR>(p, a, ((R + 16 * 32 - 1) / (16 * 32)) * 32, st);
  }
  // KT = 16 slots of nt rings: the polar caps (sin theta < kPoleSin, fewer than 0.05 R rings at
  // either end of an equiangular grid) fit in the first and last slot because nt >= R/16.
  if (R <= kFwdChunk) return launch_fwd<16, NB, 0, PAIR>(p, a, ((R + 16 * 32 - 1) / (16 * 32)) * 32, st);
  // R > kFwdChunk: the rings are split into the two polar caps (difference form throughout) and
  // interior chunks of at most kFwdChunk rings (plain form); each launch writes a partial result
  // that a fixed-order sum turns into flm.
  if (!a0.part) return cudaErrorInvalidValue;
  const long long part_elems = (long long)a.nsig * a.nN * p.L * a.flm_ld;
  int q = 0;
  cudaError_t e;
  // threads per CTA: KT * nt >= rows and nt <= rows (the last slot holds the last nt rings)
  auto nt_for = [](int rows, int kt) { return min(128, ((rows + kt - 1) / kt + 31) / 32 * 32); };
  a.part = a0.part;
  a.row0 = p.ring0; a.nrows = p.cap_n - p.ring0; a.part_off = part_elems * q++;
  if ((e = launch_fwd<4, NB, 1, PAIR>(p, a, nt_for(a.nrows, 4), st)) != cudaSuccess) return e;
  a.row0 = p.cap_s; a.nrows = p.ring0 + R - p.cap_s; a.part_off = part_elems * q++;
  if ((e = launch_fwd<4, NB, 1, PAIR>(p, a, nt_for(a.nrows, 4), st)) != cudaSuccess) return e;
  const int interior = p.cap_s - p.cap_n;
  const int nchunk = (interior + kFwdChunk - 1) / kFwdChunk;
  for (int c = 0; c < nchunk; ++c) {           // chunks of nearly equal size
    const int lo = p.cap_n + (int)((long long)interior * c / nchunk);
    const int hi = p.cap_n + (int)((long long)interior * (c + 1) / nchunk);
    a.row0 = lo; a.nrows = hi - lo; a.part_off = part_elems * q++;
    if ((e = launch_fwd<16, NB, 2, PAIR>(p, a, nt_for(a.nrows, 16), st)) != cudaSuccess) return e;
  }
  if (q != p.fwd_parts) return cudaErrorInvalidValue;
  // the orders of this launch: |m| in [(rank0 + 1) / 2, (rank0 + nrank + 1) / 2), or
  // m in [rank0, rank0 + nrank) for real-signal plans
  const int mlo = a.mpos ? a.rank0 : (a.rank0 + 1) / 2;
  const int mhi = a.mpos ? a.rank0 + a.nrank : (a.rank0 + a.nrank + 1) / 2;
  return launch_sum_parts(p, a0.part, a0.flm, a.nsig, q, mlo, mhi, a.flm_ld, a.flm_c0, st);
}

bool paired(const Plan& p) { return paired_plan(p); }

}  // namespace

namespace {

cudaError_t launch_theta_inverse_rings(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (p.mrec) return launch_theta_inverse_mrec(p, a, st);
  if (a.dtab) return launch_theta_inverse_pre(p, a, st);
  if (p.precision == S2GB_FP32) return p.tc32 ? launch_theta_inverse_tc32(p, a, st) : launch_theta_inverse_f32(p, a, st);
  if (p.tc) return launch_theta_inverse_tc(p, a, st);
  if (paired(p)) {
    if (a.nsig >= 2) return launch_inv_nb<2, true>(p, a, st);
    return launch_inv_nb<1, true>(p, a, st);
  }
  if (a.nsig >= 4) return launch_inv_nb<4, false>(p, a, st);
  if (a.nsig >= 2) return launch_inv_nb<2, false>(p, a, st);
  return launch_inv_nb<1, false>(p, a, st);
}

cudaError_t launch_theta_forward_rings(const Plan& p, const FwdArgs& a, cudaStream_t st) {
  if (p.mrec) return launch_theta_forward_mrec(p, a, st);
  if (a.dtab) return launch_theta_forward_pre(p, a, st);
  if (p.precision == S2GB_FP32) return launch_theta_forward_f32(p, a, st);
  // contraction on the tensor cores: one cluster per order (with no recursion rings -- MWSS at
  // L = 1 -- the FMA-pipe kernel writes the zero sums that the pole kernel then adds to)
  if (p.tc && p.nint > 0 && p.nint <= kFwdChunk) {
    FwdArgs b = a;
    b.row0 = p.ring0;
    b.nrows = p.nint;
    b.part = nullptr;
    b.part_off = 0;
    return launch_theta_forward_tc(p, b, st);
  }
  if (paired(p)) {
    if (a.nsig >= 2 && p.nint <= 1024) return launch_fwd_nb<2, true>(p, a, st);
    return launch_fwd_nb<1, true>(p, a, st);
  }
  if (a.nsig >= 4 && p.nint <= 1024) return launch_fwd_nb<4, false>(p, a, st);
  if (a.nsig >= 2) return launch_fwd_nb<2, false>(p, a, st);
  return launch_fwd_nb<1, false>(p, a, st);
}

}  // namespace

// The recursion kernels over the rings [ring0, ring0 + nint), then the pole rings the plan hands
// to the exact pole kernels (MWSS; MW with the order recursion).
cudaError_t launch_theta_inverse(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (a.nrank <= 0) return cudaSuccess;             // no orders in range: nothing to launch
  const cudaError_t e = launch_theta_inverse_rings(p, a, st);
  if (e != cudaSuccess || (p.pole_n < 0 && p.pole_s < 0)) return e;
  return launch_pole_inverse(p, a, st);
}

cudaError_t launch_theta_forward(const Plan& p, const FwdArgs& a, cudaStream_t st) {
  if (a.nrank <= 0) return cudaSuccess;
  const cudaError_t e = launch_theta_forward_rings(p, a, st);
  if (e != cudaSuccess || (p.pole_n < 0 && p.pole_s < 0)) return e;
  return launch_pole_forward(p, a, st);
}

}  // namespace s2gb
