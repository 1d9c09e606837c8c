// Float32 theta stages (the mixed-precision path).  Same recursion, layouts and thread mapping as
// the float64 kernels in theta_kernels.cu, with:
//   * starting values computed in float64 (double-double logarithms, as in the float64 path) and
//     converted to a float mantissa plus an integer exponent;
//   * the recursion and the products in float32 (coefficients rounded once from the double-double
//     tables), dead-chain bookkeeping every 2 steps because of float32's narrow exponent range;
//   * compensated accumulation: the inverse folds blocks of 32 degrees into a (hi, lo) pair with
//     Knuth's two-sum; the forward reduces its per-thread partial sums across the warp with a
//     reduce-scatter whose top two levels use two-sum, and across warps in float64;
//   * once all chains of a warp are live, the exponent bookkeeping stops (a live chain stays live).
#include "theta_f32.cuh"

namespace s2gb {

namespace {
using namespace theta;

constexpr int kChunk32 = 32;

// ------------------------------------------------------------------------------------------ inverse
// Accumulation: each thread sums 32 degrees (one staged chunk) per (ring, signal) in float32
// registers, then folds that block sum into a compensated (hi, lo) pair kept in shared memory
// (acc: [KT * NB slots][hi, lo][threads]) with Knuth's two-sum.  Keeping the pairs in shared memory
// leaves registers for up to 8 signals per CTA, over which the recursion is shared.
template <int KT, int NB, bool DIFF>
__device__ __forceinline__ void inverse_body_f32(const InvArgs& a, int m, int ni, int tile, int l0,
                                                 float2* __restrict__ hs, float* __restrict__ cs,
                                                 float2* __restrict__ acc) {
  const int L = a.L, T = 2 * L - 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mi = m + L - 1;
  const int sig0 = blockIdx.z * NB;
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  const float* coef_m = a.coef32 + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStep;

  float x[KT], y[KT], v[KT];
  int E[KT], tt[KT];
  bool north[KT];
  unsigned nmask[KT];
  float2 blk[KT][NB];
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    const int t = a.ring0 + tile * KT * nt + i * nt + tid;
    tt[i] = t;
    if (t < a.nring) {
      const RingData rd = a.ring[t];
      seed_value_f32(sd, rd, x[i], E[i]);
      v[i] = a.v32[t];
      north[i] = rd.north;
    } else {
      x[i] = 0.0f; E[i] = 0; v[i] = 0.0f; north[i] = true;
    }
    nmask[i] = north[i] ? 0x80000000u : 0u;
    y[i] = DIFF ? x[i] : 0.0f;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      blk[i][b] = make_float2(0.f, 0.f);
      acc[(2 * (i * NB + b)) * nt + tid] = make_float2(0.f, 0.f);
      acc[(2 * (i * NB + b) + 1) * nt + tid] = make_float2(0.f, 0.f);
    }
  }

  // once every chain of the warp is live (|d| >= 2^-90 in float32 range) it stays live: the
  // exponent bookkeeping and the live-mask votes stop
  bool all_live = false;
  unsigned live = 0;
  const double* scale = a.scale + (size_t)ni * L;
  for (int jc = l0; jc < L; jc += kChunk32) {
    __syncthreads();
    for (int q = tid; q < kChunk32 * NB; q += nt) {
      const int jj = q / NB, b = q % NB, j = jc + jj, sig = sig0 + b;
      float2 h = make_float2(0.f, 0.f);
      if (j < L && sig < a.nsig) {
        h = reinterpret_cast<const float2*>(a.flm)[((size_t)(sig * a.nN + ni) * L + j) * a.flm_ld + m + a.flm_c0];
        if (a.mpos && m == 0) h.y = 0.f;      // real signals: flm(l, 0) is real
        const float s = (float)scale[j];
        h.x *= s; h.y *= s;
      }
      hs[q] = h;
    }
    for (int q = tid; q < kChunk32 * kCoefPerStep; q += nt) {
      const int j = jc + q / kCoefPerStep;
      cs[q] = (j < L) ? coef_m[(size_t)jc * kCoefPerStep + q] : 0.0f;
    }
    __syncthreads();
    const int jend = min(kChunk32, L - jc);
    for (int j8 = 0; j8 < jend; j8 += 8) {
      if (!all_live) {
        live = 0;
#pragma unroll
        for (int i = 0; i < KT; ++i) live |= (__any_sync(0xffffffffu, E[i] == 0) ? 1u : 0u) << i;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int jj = j8 + u;
        if (jj < jend) {
          float2 h[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) h[b] = hs[jj * NB + b];
#pragma unroll
          for (int i = 0; i < KT; ++i) {
            if ((live >> i) & 1u) {
              const float xl = (E[i] == 0) ? x[i] : 0.0f;
#pragma unroll
              for (int b = 0; b < NB; ++b) {
                blk[i][b].x = fmaf(xl, h[b].x, blk[i][b].x);
                blk[i][b].y = fmaf(xl, h[b].y, blk[i][b].y);
              }
            }
          }
          if (jc + jj < L - 1) {
            const float* cp = cs + jj * kCoefPerStep;
            const StepCoef32 c = {cp[0], cp[1], cp[2], cp[3], cp[4], cp[5]};
#pragma unroll
            for (int i = 0; i < KT; ++i) step_f32<DIFF>(x[i], y[i], v[i], nmask[i], north[i], c);
          }
        }
        if ((u & 1) && !all_live) {
#pragma unroll
          for (int i = 0; i < KT; ++i) renorm_f32(x[i], y[i], E[i]);
          live = 0;   // chains may have come alive: refresh the warp-uniform mask
          bool mine = true;
#pragma unroll
          for (int i = 0; i < KT; ++i) {
            live |= (__any_sync(0xffffffffu, E[i] == 0) ? 1u : 0u) << i;
            mine = mine && E[i] == 0;
          }
          all_live = __all_sync(0xffffffffu, mine);
        }
      }
    }
    // fold the chunk's block sums into the compensated (hi, lo) pairs
#pragma unroll
    for (int i = 0; i < KT; ++i) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        float2& hi = acc[(2 * (i * NB + b)) * nt + tid];
        float2& lo = acc[(2 * (i * NB + b) + 1) * nt + tid];
        float2 h2 = hi, l2 = lo;
        float s, e;
        two_sum_f(h2.x, blk[i][b].x, s, e); h2.x = s; l2.x += e;
        two_sum_f(h2.y, blk[i][b].y, s, e); h2.y = s; l2.y += e;
        hi = h2; lo = l2;
        blk[i][b] = make_float2(0.f, 0.f);
      }
    }
  }

#pragma unroll
  for (int i = 0; i < KT; ++i) {
    if (tt[i] < a.nring) {
      const long long col = a.m_mod ? (m >= 0 ? m : m + a.mmod) : mi;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int sig = sig0 + b;
        if (sig < a.nsig) {
          const float2 hi = acc[(2 * (i * NB + b)) * nt + tid], lo = acc[(2 * (i * NB + b) + 1) * nt + tid];
          float2* o = reinterpret_cast<float2*>(a.out) + (size_t)(sig * a.nN + ni) * a.s_sig +
                      tt[i] * a.s_t + col * a.s_m;
          *o = make_float2(hi.x + lo.x, hi.y + lo.y);
        }
      }
    }
  }
}

template <int KT, int NB>
__global__ void __launch_bounds__(128) theta_inverse_kernel_f32(InvArgs a, int ntiles) {
  __shared__ float2 hs[kChunk32 * NB];
  __shared__ float cs[kChunk32 * kCoefPerStep];
  extern __shared__ float2 acc_smem[];            // [KT * NB][2][blockDim.x]
  const int L = a.L;
  const int rank = a.rank0 + (int)(blockIdx.x / ntiles), tile = blockIdx.x % ntiles;
  const int m = a.mpos ? rank : m_of_rank(rank);
  const int ni = blockIdx.y;
  const int l0 = a.seed[(size_t)ni * (2 * L - 1) + m + L - 1].l0;
  const int t_lo = a.ring0 + tile * KT * blockDim.x, t_hi = min(a.nring, t_lo + KT * (int)blockDim.x) - 1;
  const bool diff = a.ring[t_lo].diff || a.ring[t_hi].diff;
  if (diff) inverse_body_f32<KT, NB, true>(a, m, ni, tile, l0, hs, cs, acc_smem);
  else inverse_body_f32<KT, NB, false>(a, m, ni, tile, l0, hs, cs, acc_smem);
}

// ------------------------------------------------------------------------------------------ forward
// Warp reduce-scatter of 32 partial sums: lane l ends with slot l as an unevaluated (hi, lo) pair.
// The first three levels (sums of up to 8 lanes) add in plain float32; the top two levels, where
// the partial sums and hence the rounding errors are largest, use Knuth's two-sum and carry the
// error terms.
__device__ __forceinline__ void warp_reduce_scatter32_f(float (&h)[32], float& oh, float& ol) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 16; w >= 4; w >>= 1) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int s = 0; s < w; ++s) {
      const float send = up ? h[s] : h[s + w];
      const float keep = up ? h[s + w] : h[s];
      h[s] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  float l[2] = {0.f, 0.f};
#pragma unroll
  for (int w = 2; w >= 1; w >>= 1) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int s = 0; s < w; ++s) {
      const float sh = up ? h[s] : h[s + w];
      const float sl = up ? l[s] : l[s + w];
      const float kh = up ? h[s + w] : h[s];
      const float kl = up ? l[s + w] : l[s];
      const float rh = __shfl_xor_sync(0xffffffffu, sh, w);
      const float rl = __shfl_xor_sync(0xffffffffu, sl, w);
      float sum, err;
      two_sum_f(kh, rh, sum, err);
      h[s] = sum;
      l[s] = kl + rl + err;
    }
  }
  oh = h[0];
  ol = l[0];
}

template <int KT, int NB, int PAT>
__global__ void __launch_bounds__(256) theta_forward_kernel_f32(FwdArgs a) {
  constexpr int JR = 16 / NB;
  extern __shared__ double smem64[];
  const int L = a.L, T = 2 * L - 1;
  const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nt >> 5;
  const int rows = KT * nt;
  double* red = smem64;                                            // [2][nwarps][32]
  float2* gs = reinterpret_cast<float2*>(red + 2 * nwarps * 32);  // [NB][rows]
  float* vs = reinterpret_cast<float*>(gs + NB * rows);           // [rows]

  const int m = a.mpos ? a.rank0 + (int)blockIdx.x : m_of_rank(a.rank0 + (int)blockIdx.x);
  const int mi = m + L - 1;
  const int ni = blockIdx.y;
  const int sig0 = blockIdx.z * NB;
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  const int l0 = sd.l0;
  const double* scale = a.scale + (size_t)ni * L;

  for (int q = tid; q < NB * min(l0, L); q += nt) {
    const int b = q / min(l0, L), j = q % min(l0, L), sig = sig0 + b;
    if (sig < a.nsig)
      reinterpret_cast<float2*>(a.flm)[((size_t)(sig * a.nN + ni) * L + j) * a.flm_ld + m + a.flm_c0] = make_float2(0.f, 0.f);
  }
  if (l0 >= L) return;

  const long long col = a.m_mod ? (m >= 0 ? m : m + a.mmod) : mi;
  const int R = a.nrows, r0 = a.row0;    // rings [r0, r0 + R) (one launch covers every ring)
  for (int q = tid; q < NB * rows; q += nt) {
    const int b = q / rows, pos = q % rows, sig = sig0 + b;
    bool act;
    const int t = r0 + ring_of<KT>(pos / nt, pos % nt, nt, R, act);
    float2 g = make_float2(0.f, 0.f);
    if (act && sig < a.nsig) {
      g = reinterpret_cast<const float2*>(a.g)[(size_t)(sig * a.nN + ni) * a.s_sig + t * a.s_t + col * a.s_m];
      if (a.use_nu) { const float w = (float)a.nu[t]; g.x *= w; g.y *= w; }
    }
    gs[q] = g;
  }
  for (int pos = tid; pos < rows; pos += nt) {
    bool act;
    const int t = r0 + ring_of<KT>(pos / nt, pos % nt, nt, R, act);
    vs[pos] = act ? a.v32[t] : 0.0f;
  }
  __syncthreads();

  float x[KT], y[KT];
  int E[KT];
  bool north[KT];
  unsigned nmask[KT];
#pragma unroll
  for (int i = 0; i < KT; ++i) {
    bool act;
    const int t = r0 + ring_of<KT>(i, tid, nt, R, act);
    if (act) {
      const RingData rd = a.ring[t];
      seed_value_f32(sd, rd, x[i], E[i]);
      north[i] = rd.north;
    } else {
      x[i] = 0.0f; E[i] = 0; north[i] = true;
    }
    nmask[i] = north[i] ? 0x80000000u : 0u;
    const bool dslot = (PAT == 1) || i == 0 || i == KT - 1;
    y[i] = dslot ? x[i] : 0.0f;
  }

  const float* coef_m = a.coef32 + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStep;
  int buf = 0;
  // once every chain of the warp is live it stays live: the bookkeeping and votes stop
  bool all_live = false;
  unsigned live = 0;
  for (int j0 = l0; j0 < L; j0 += JR) {
    float ph[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) ph[s] = 0.f;
    if (!all_live) {
      live = 0;
#pragma unroll
      for (int i = 0; i < KT; ++i) live |= (__any_sync(0xffffffffu, E[i] == 0) ? 1u : 0u) << i;
    }
#pragma unroll
    for (int jr = 0; jr < JR; ++jr) {
      const int j = j0 + jr;
      if (j < L) {
#pragma unroll
        for (int i = 0; i < KT; ++i) {
          if ((live >> i) & 1u) {
            const float xl = (E[i] == 0) ? x[i] : 0.0f;
            const int pos = i * nt + tid;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              const float2 g = gs[b * rows + pos];
              ph[jr * 2 * NB + 2 * b] = fmaf(xl, g.x, ph[jr * 2 * NB + 2 * b]);
              ph[jr * 2 * NB + 2 * b + 1] = fmaf(xl, g.y, ph[jr * 2 * NB + 2 * b + 1]);
            }
          }
        }
        if (j < L - 1) {
          const float* cp = coef_m + (size_t)j * kCoefPerStep;
          const float2 c01 = __ldg(reinterpret_cast<const float2*>(cp));
          const float2 c23 = __ldg(reinterpret_cast<const float2*>(cp) + 1);
          const float2 c45 = __ldg(reinterpret_cast<const float2*>(cp) + 2);
          const StepCoef32 c = {c01.x, c01.y, c23.x, c23.y, c45.x, c45.y};
#pragma unroll
          for (int i = 0; i < KT; ++i) {
            const float v = vs[i * nt + tid];
            const bool dslot = (PAT == 1) || i == 0 || i == KT - 1;
            if (dslot) step_f32<true>(x[i], y[i], v, nmask[i], north[i], c);
            else step_f32<false>(x[i], y[i], v, nmask[i], north[i], c);
          }
        }
      }
      if (((jr & 1) || jr == JR - 1) && !all_live) {
#pragma unroll
        for (int i = 0; i < KT; ++i) renorm_f32(x[i], y[i], E[i]);
        live = 0;   // chains may have come alive: refresh the warp-uniform mask
        bool mine = true;
#pragma unroll
        for (int i = 0; i < KT; ++i) {
          live |= (__any_sync(0xffffffffu, E[i] == 0) ? 1u : 0u) << i;
          mine = mine && E[i] == 0;
        }
        all_live = __all_sync(0xffffffffu, mine);
      }
    }
    float oh, ol;
    warp_reduce_scatter32_f(ph, oh, ol);
    red[(buf * nwarps + warp) * 32 + lane] = (double)oh + (double)ol;
    __syncthreads();
    if (warp == 0) {
      double tot = red[(buf * nwarps) * 32 + lane];
      for (int w = 1; w < nwarps; ++w) tot += red[(buf * nwarps + w) * 32 + lane];
      const int jr = lane / (2 * NB), b = (lane / 2) % NB, reim = lane & 1;
      const int j = j0 + jr, sig = sig0 + b;
      if (j < L && sig < a.nsig) {
        float* o = reinterpret_cast<float*>(
            reinterpret_cast<float2*>(a.flm) + ((size_t)(sig * a.nN + ni) * L + j) * a.flm_ld + m + a.flm_c0);
        o[reim] = (float)(tot * scale[j]);
      }
    }
    buf ^= 1;
  }
}

template <int KT, int NB>
cudaError_t launch_inv32(const Plan& p, const InvArgs& a, cudaStream_t st) {
  const int nt = 128;
  const int ntiles = (a.nring - a.ring0 + KT * nt - 1) / (KT * nt);
  if (ntiles == 0) return cudaSuccess;          // no rings for the recursion (MWSS, L = 1)
  const size_t smem = sizeof(float2) * 2 * KT * NB * nt;
  auto kern = theta_inverse_kernel_f32<KT, NB>;
  cudaError_t e = set_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nrank * ntiles, a.nN, (a.nsig + NB - 1) / NB);
  kern<<<grid, nt, smem, st>>>(a, ntiles);
  return launched();
}

template <int NB>
cudaError_t launch_inv32_nb(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (a.nring - a.ring0 <= 128) return launch_inv32<1, NB>(p, a, st);
  if (a.nring - a.ring0 <= 512) return launch_inv32<2, NB>(p, a, st);
  return launch_inv32<4, NB>(p, a, st);
}

template <int KT, int NB, int PAT>
cudaError_t launch_fwd32(const Plan& p, const FwdArgs& a, int nt, cudaStream_t st) {
  const int rows = KT * nt;
  const size_t smem = sizeof(double) * 2 * (nt / 32) * 32 + sizeof(float2) * NB * rows + sizeof(float) * rows;
  auto kern = theta_forward_kernel_f32<KT, NB, PAT>;
  cudaError_t e = set_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nrank, a.nN, (a.nsig + NB - 1) / NB);
  kern<<<grid, nt, smem, st>>>(a);
  return launched();
}

template <int NB>
cudaError_t launch_fwd32_nb(const Plan& p, const FwdArgs& a0, cudaStream_t st) {
  const int R = p.nint;    // rings of the recursion (float32 plans have nint <= kFwdChunk)
  FwdArgs a = a0;
  a.row0 = p.ring0;
  a.nrows = R;
  if (R <= 128) return launch_fwd32<1, NB, 1>(p, a, R > 32 ? ((R + 31) / 32) * 32 : 32, st);
  if (R <= 256) return launch_fwd32<2, NB, 1>(p, a, 128, st);
  if (R <= 512) return launch_fwd32<4, NB, 0>(p, a, 128, st);
  if (R <= 1024) return launch_fwd32<8, NB, 0>(p, a, 128, st);
  // up to 2048 rings: 8 rings per thread and up to 256 threads (the polar caps fit in the first and
  // last slot of nt >= R/8 rings); more threads per SM than 16 rings per thread would allow
  const int nt = ((R + 8 * 32 - 1) / (8 * 32)) * 32;
  if (nt > 256) return cudaErrorInvalidConfiguration;
  return launch_fwd32<8, NB, 0>(p, a, nt, st);
}

}  // namespace

cudaError_t launch_theta_inverse_f32(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (a.nsig >= 8) return launch_inv32_nb<8>(p, a, st);
  if (a.nsig >= 4) return launch_inv32_nb<4>(p, a, st);
  if (a.nsig >= 2) return launch_inv32_nb<2>(p, a, st);
  return launch_inv32_nb<1>(p, a, st);
}

cudaError_t launch_theta_forward_f32(const Plan& p, const FwdArgs& a, cudaStream_t st) {
  if (a.nsig >= 8 && p.nint <= 1024) return launch_fwd32_nb<8>(p, a, st);
  if (a.nsig >= 4) return launch_fwd32_nb<4>(p, a, st);
  if (a.nsig >= 2) return launch_fwd32_nb<2>(p, a, st);
  return launch_fwd32_nb<1>(p, a, st);
}

}  // namespace s2gb
