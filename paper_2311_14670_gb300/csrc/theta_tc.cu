// Inverse theta stage (Sec. 4.1, Eq. disc_ish_expanded; interleaved as in Sec. 4.4) with the
// contraction over the degree on the tensor cores.
//
// For one order m the stage is a product: out[t][c] = sum_l x_l(theta_t) h'_l[c], the ring x degree
// matrix of d-functions (generated on the fly by the float64 recursion of theta_kernels.cu, one
// chain per thread) times a degree x column block of coefficients (c = real and imaginary part of
// each signal slot).  On GB300 the float64 pipe (2 lanes per SM and clock) is the scarce unit: the
// recursion needs 2 of its FMAs per element, the contraction 2 per element and signal.  Here the
// recursion alone stays on the float64 pipe; the contraction runs as exact integer arithmetic on
// the float16 tensor cores, after the splitting of the Ozaki scheme (Ozaki, Ogita, Oishi, Rump,
// Numer. Algorithms 59, 2012; on float16 tensor cores: Mukunoki, Ozaki, Ogita, Imamura, 2020):
//
//   * every recursion value becomes a fixed-point integer qa = trunc(x 2^(55 - rho_l)), with rho_l a
//     power-of-two bound of |x| at degree l (|u^l| <= 1/gamma_l for the block-normalised values,
//     |d| <= 1 in the difference form), and every coefficient qh = trunc(h' 2^(55 - eps_c)) with one
//     exponent eps_c per column (the largest over the degrees of the CTA's order);
//     the scale 2^rho_l moves into the coefficient of degree l, so the product is unchanged;
//   * |q| < 2^54 is written in 7 balanced base-256 digits in [-128, 127] (adding 0x80 to every
//     byte of the two's complement integer and subtracting it again digit by digit), each digit
//     exact in float16;
//   * one tcgen05.mma per digit i of the d-values multiplies the i-th digit matrix (128 rings x
//     16 degrees) by the digits j <= 6 - i of the coefficients (16 degrees x 8 columns each) and
//     accumulates in float32 in Tensor Memory.  Every product is an integer below 2^14 in
//     magnitude, so up to 1024 degrees sum exactly below 2^24; the accumulators are read back every
//     1024 degrees (and at the end), converted to integers, combined with the weights
//     256^(12 - i - j) in 64-bit integers and added in float64.  Digit products with i + j > 6
//     are dropped: their weight is below 2^-48 of the leading ones, under the rounding of the
//     float64 recursion.
//
// Mapping: CTA = (order rank, tile of 128 rings, n, batch group); thread tid = ring = TMEM lane.
// Per chunk of 16 degrees each thread advances its chain 16 steps, writing its 7 digit rows into
// shared memory (K-major 8 x 16-byte core matrices); 64 threads write the coefficient digits; after
// a CTA barrier one thread issues the 7 MMAs and commits them to the chunk's mbarrier.  Three
// stages of operand buffers let the recursion of the next chunks overlap the tensor cores.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tc_common.cuh"
#include "theta_common.cuh"

// Status of the tensor-core kernels on this device: 0, or the first tc::kStatus* code recorded by a
// kernel whose bounded wait ran out (read and cleared by s2gb_device_status).
__device__ int g_s2gb_device_status;

namespace s2gb {

namespace {
using namespace theta;

constexpr int kTcRings = 128;        // rings per CTA = MMA M = TMEM lanes
constexpr int kTcK = 16;             // degrees per chunk = MMA K (float16)
constexpr int kTcStages = 3;         // operand stages in flight
constexpr int kDigits = 7;           // balanced base-256 digits per operand
constexpr int kDrainChunks = 64;     // 1024 degrees: |sum of digit products| <= 1024 * 2^14 = 2^24
constexpr int kATileBytes = kTcRings * kTcK * 2;        // one digit matrix (4 KiB)
constexpr int kAStageBytes = kDigits * kATileBytes;     // 28 KiB

// Columns of the accumulator of A-digit i: the B digits j = 0 .. 6 - i of C columns each, padded to
// a multiple of 16 (the MMA's N granularity at M = 128; the padding rows are the zero digit 7).
template <int C>
struct TcCols {
  static constexpr int n(int i) { return ((C * (kDigits - i) + 15) / 16) * 16; }
  static constexpr int off(int i) { return i == 0 ? 0 : off(i - 1) + n(i - 1); }
  static constexpr int total = off(kDigits - 1) + n(kDigits - 1);
  static constexpr int alloc = total <= 32 ? 32 : total <= 64 ? 64 : total <= 128 ? 128 : total <= 256 ? 256 : 512;
};

template <int C>
struct TcSmem {
  static constexpr int kBRows = 8 * C;                    // digits 0..7 (7: zero) x C columns
  static constexpr int kBStageBytes = kBRows * kTcK * 2;
  static constexpr int a_off = 0;
  static constexpr int b_off = a_off + kTcStages * kAStageBytes;
  static constexpr int cs_off = b_off + kTcStages * kBStageBytes;
  static constexpr int bar_off = cs_off + 2 * kTcK * kCoefPerStepN * 8;
  static constexpr int misc_off = bar_off + kTcStages * 8;
  static constexpr int bytes = misc_off + 4 * (C + 4);
};

// Byte offset of element (row, k) in a K-major operand tile of 16 columns: 8-row x 16-byte core
// matrices, the two K halves 128 bytes apart (LBO), row groups 256 bytes apart (SBO).
__device__ __forceinline__ int kmajor_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// trunc(|x| 2^(55 - rho)) with the sign of x, plus 0x0080808080808080: byte p (p = 0..6) of the
// result is the balanced base-256 digit of weight 256^p, offset by 128.  Needs |x| < 2^(rho - 1).
// Zero and subnormal x give the digits of 0.
__device__ __forceinline__ uint2 offset_digits(double x, int rho) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7ffu);
  const uint32_t sh = ex == 0 ? 64u : (uint32_t)(1023 + rho - ex);
  const uint64_t m = ((((uint64_t)((hi & 0xfffffu) | 0x100000u)) << 32) | lo) << 3;   // 56 bits
  uint64_t q;
  asm("shr.b64 %0, %1, %2;" : "=l"(q) : "l"(m), "r"(sh));
  const uint64_t neg = (uint64_t)(int64_t)((int32_t)hi >> 31);
  q = ((q ^ neg) - neg) + 0x0080808080808080ull;
  return make_uint2((uint32_t)q, (uint32_t)(q >> 32));
}

// The float16 pair (digit of element 0, digit of element 1) at byte p (0..3) of the words w0, w1.
__device__ __forceinline__ uint32_t digit_pair(uint32_t w0, uint32_t w1, int p) {
  uint32_t r = __byte_perm(w0, w1, (uint32_t)(p | (p << 4) | ((p + 4) << 8) | ((p + 4) << 12)));
  r = (r & 0x00ff00ffu) | 0x64006400u;            // float16 1024 + byte, exact
  __half2 h = *reinterpret_cast<__half2*>(&r);
  h = __hsub2(h, __floats2half2_rn(1152.0f, 1152.0f));   // byte - 128, exact
  return *reinterpret_cast<uint32_t*>(&h);
}

// Digit i (0 = most significant, byte 6) of an offset_digits result as a float16 bit pattern.
__device__ __forceinline__ unsigned short digit_half(uint2 q, int i) {
  const int p = 6 - i;
  const uint32_t byte = ((p >= 4 ? q.y >> (8 * (p - 4)) : q.x >> (8 * p)) & 0xffu);
  return __half_as_ushort(__float2half_rn((float)((int)byte - 128)));
}

__device__ __forceinline__ void set_status(int code) { atomicCAS(&g_s2gb_device_status, 0, code); }

// Coefficient h'_{j,b} of signal slot b at degree j (times 2^rho_j), both parts.
template <int NB, bool PAIR, bool DIFF>
__device__ __forceinline__ double2 coef_scaled(const InvArgs& a, const double* coef_m, const double* scale,
                                               int j, int b, int sig0, int ni, int m, int n, int L) {
  const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
  double2 h = make_double2(0.0, 0.0);
  if (sl.sig_off >= 0) {
    h = reinterpret_cast<const double2*>(a.flm)[((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0];
    if (a.mpos && m == 0) h.y = 0.0;
    const double* c = coef_m + (size_t)j * kCoefPerStepN;
    const int rho = DIFF ? 2 : exp_of(c[9]) + 2;
    const double s = sl.sign * (DIFF ? scale[j] : scale[j] * c[3]) * pow2i(rho);
    h.x *= s;
    h.y *= s;
  }
  return h;
}

template <int NB, bool PAIR, bool DIFF>
__device__ __forceinline__ void tc_inverse_body(const InvArgs& a, int m, int ni, int n, int tile, int l0,
                                                unsigned char* smem) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  constexpr int C = 2 * NBX;
  using Cols = TcCols<C>;
  using Sm = TcSmem<C>;
  const int L = a.L, T = 2 * L - 1;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mi = m + L - 1;
  const int sig0 = blockIdx.z * NB;

  unsigned char* sA = smem + Sm::a_off;
  unsigned char* sB = smem + Sm::b_off;
  double* cs = reinterpret_cast<double*>(smem + Sm::cs_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sm::bar_off);
  int* eps_s = reinterpret_cast<int*>(smem + Sm::misc_off);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(eps_s + C);
  int* abort_s = reinterpret_cast<int*>(eps_s + C + 1);

  const double* coef_m = a.coef + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStepN;
  const double* scale = a.scale + (size_t)ni * L;

  // ---- set-up: barriers, Tensor Memory, zero digit rows, column exponents
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) tc::mbar_init(tc::smem_addr(&bars[s]), 1);
    tc::mbar_init_fence();
    *abort_s = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_slot), Cols::alloc);
  for (int q = tid; q < kTcStages * Sm::kBStageBytes / 16; q += kTcRings)
    reinterpret_cast<uint4*>(sB)[q] = make_uint4(0, 0, 0, 0);
  if (tid < C) eps_s[tid] = -100000;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const int ndeg = L - l0;
  for (int q = tid; q < ndeg * NBX; q += kTcRings) {
    const int j = l0 + q / NBX, b = q % NBX;
    const double2 h = coef_scaled<NB, PAIR, DIFF>(a, coef_m, scale, j, b, sig0, ni, m, n, L);
    if (h.x != 0.0) atomicMax(&eps_s[2 * b], exp_of(h.x));
    if (h.y != 0.0) atomicMax(&eps_s[2 * b + 1], exp_of(h.y));
  }
  // coefficients of the first chunk
  for (int q = tid; q < kTcK * kCoefPerStepN; q += kTcRings) {
    const int j = l0 + q / kCoefPerStepN;
    cs[q] = (j < L) ? coef_m[(size_t)l0 * kCoefPerStepN + q] : 0.0;
  }
  __syncthreads();
  // column exponents: |h'| < 2^(eps_c - 1) (an all-zero column keeps eps_c = 2)
  auto col_eps = [&](int c) { const int e = eps_s[c]; return (e < -2000 ? 0 : e) + 2; };
  int eps[C];
#pragma unroll
  for (int c = 0; c < C; ++c) eps[c] = col_eps(c);

  // ---- the chain of this thread's ring
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  const int t = a.ring0 + tile * kTcRings + tid;
  double x = 0.0, y = 0.0, v = 0.0;
  int E = 0;
  bool north = true;
  if (t < a.nring) {
    const RingData rd = a.ring[t];
    seed_value(sd, rd, x, E);
    v = rd.v;
    north = rd.north;
  }
  const unsigned nmask = north ? 0x80000000u : 0u;

  double acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.0;

  const int nchunks = (ndeg + kTcK - 1) / kTcK;
  int since_reset = 0;
  bool ok = true;
  const uint32_t sA_addr = tc::smem_addr(sA), sB_addr = tc::smem_addr(sB);
  for (int k = 0; k < nchunks; ++k) {
    const int s = k % kTcStages;
    const int jc = l0 + k * kTcK;
    const double* csk = cs + (k & 1) * kTcK * kCoefPerStepN;
    // prefetch: the coefficients of the next chunk, and this chunk's h' for the B digits
    double cpre[2] = {0.0, 0.0};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int q = tid + r * kTcRings;
      const int j = jc + kTcK + q / kCoefPerStepN;
      if (q < kTcK * kCoefPerStepN && j < L) cpre[r] = coef_m[(size_t)(jc + kTcK) * kCoefPerStepN + q];
    }
    double2 hpre = make_double2(0.0, 0.0);
    const int hb = tid % NBX, hj = jc + tid / NBX;
    if (tid < kTcK * NBX && hj < L) hpre = coef_scaled<NB, PAIR, DIFF>(a, coef_m, scale, hj, hb, sig0, ni, m, n, L);

    // the stage's previous MMAs (chunk k - 3) must be complete before its buffers are rewritten
    if (k >= kTcStages && !tc::mbar_wait(tc::smem_addr(&bars[s]), (uint32_t)((k / kTcStages - 1) & 1))) {
      set_status(tc::kStatusMmaWait);
      *abort_s = 1;
    }

    unsigned char* aStage = sA + s * kAStageBytes;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      uint32_t w[kDigits][4];
      const bool live = __any_sync(0xffffffffu, E == 0);
      uint2 q0 = make_uint2(0, 0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int jj = g * 8 + u, j = jc + jj;
        const StepN c = stepn_at(csk + jj * kCoefPerStepN);
        if (live) {
          const double xl = (E == 0 && j < L) ? x : 0.0;
          const int rho = DIFF ? 2 : exp_of(c.ig) + 2;
          const uint2 q = offset_digits(xl, rho);
          if (u & 1) {
            w[0][u >> 1] = digit_pair(q0.y, q.y, 2);
            w[1][u >> 1] = digit_pair(q0.y, q.y, 1);
            w[2][u >> 1] = digit_pair(q0.y, q.y, 0);
            w[3][u >> 1] = digit_pair(q0.x, q.x, 3);
            w[4][u >> 1] = digit_pair(q0.x, q.x, 2);
            w[5][u >> 1] = digit_pair(q0.x, q.x, 1);
            w[6][u >> 1] = digit_pair(q0.x, q.x, 0);
          } else {
            q0 = q;
          }
        }
        if (j < L - 1) {
          stepn<DIFF>(x, y, v, nmask, north, c);
          if (u == kNormBlock - 1) unnormalise<DIFF>(x, y, c);
        }
      }
      renorm(x, y, E);
#pragma unroll
      for (int i = 0; i < kDigits; ++i) {
        uint4 val = live ? make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]) : make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(aStage + i * kATileBytes + kmajor_off(tid, g * 8)) = val;
      }
    }
    // B digits of this chunk: thread (degree jj, slot b) writes rows (i, 2b) and (i, 2b + 1)
    if (tid < kTcK * NBX) {
      unsigned char* bStage = sB + s * Sm::kBStageBytes;
      const int jj = tid / NBX;
      const uint2 qr = offset_digits(hpre.x, col_eps(2 * hb));
      const uint2 qi = offset_digits(hpre.y, col_eps(2 * hb + 1));
#pragma unroll
      for (int i = 0; i < kDigits; ++i) {
        *reinterpret_cast<unsigned short*>(bStage + kmajor_off(i * C + 2 * hb, jj)) = digit_half(qr, i);
        *reinterpret_cast<unsigned short*>(bStage + kmajor_off(i * C + 2 * hb + 1, jj)) = digit_half(qi, i);
      }
    }
    // the next chunk's recursion coefficients
    {
      double* csn = cs + ((k + 1) & 1) * kTcK * kCoefPerStepN;
      csn[tid] = cpre[0];
      if (tid + kTcRings < kTcK * kCoefPerStepN) csn[tid + kTcRings] = cpre[1];
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (*abort_s) { ok = false; break; }
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int i = 0; i < kDigits; ++i) {
        const uint64_t ad = tc::smem_desc(sA_addr + s * kAStageBytes + i * kATileBytes, 128, 256);
        const uint64_t bd = tc::smem_desc(sB_addr + s * Sm::kBStageBytes, 128, 256);
        tc::mma_f16(tmem + Cols::off(i), ad, bd, tc::idesc_f16_f32(kTcRings, Cols::n(i)), since_reset > 0);
      }
      tc::mma_commit(tc::smem_addr(&bars[s]));
    }
    ++since_reset;
    if (since_reset == kDrainChunks || k == nchunks - 1) {
      // read the accumulators back: integer digit sums per level i + j, combined exactly
      if (!tc::mbar_wait(tc::smem_addr(&bars[s]), (uint32_t)((k / kTcStages) & 1))) {
        set_status(tc::kStatusMmaWait);
        ok = false;
      }
      tc::fence_after_sync();
      if (__all_sync(0xffffffffu, ok)) {
        int lam[kDigits][C];
#pragma unroll
        for (int i = 0; i < kDigits; ++i)
#pragma unroll
          for (int c = 0; c < C; ++c) lam[i][c] = 0;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int i = 0; i < kDigits; ++i) {
          const int ncol = C * (kDigits - i);
#pragma unroll
          for (int q8 = 0; q8 < (C * kDigits + 7) / 8; ++q8) {
            if (q8 * 8 < ncol) {
              uint32_t r[8];
              tc::tmem_ld8(trow + (uint32_t)(Cols::off(i) + 8 * q8), r);
              tc::tmem_ld_wait();
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int col = 8 * q8 + e;
                if (col < ncol) lam[i + col / C][col % C] += __float2int_rn(__uint_as_float(r[e]));
              }
            }
          }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const long long hv = ((long long)lam[0][c] << 24) + ((long long)lam[1][c] << 16) +
                               ((long long)lam[2][c] << 8) + (long long)lam[3][c];
          const long long lv = ((long long)lam[4][c] << 16) + ((long long)lam[5][c] << 8) + (long long)lam[6][c];
          const double val = fma((double)lv, 0x1p-24, (double)hv);
          acc[c] += ldexp(val, eps[c] - 38);
        }
      }
      tc::fence_before_sync();
      since_reset = 0;
      if (!__syncthreads_and(ok)) { ok = false; break; }
    }
  }

  if (ok) {
#pragma unroll
    for (int b = 0; b < NBX; ++b) {
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      if (sl.sig_off < 0 || t >= a.nring) continue;
      const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
      double2* o = reinterpret_cast<double2*>(a.out) + (size_t)sl.sig_off * a.s_sig + t * a.s_t + col * a.s_m;
      *o = make_double2(acc[2 * b], acc[2 * b + 1]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, Cols::alloc);
  }
}

// Grid as theta_inverse_kernel: x = (rank of m) * ntiles + tile, y = n index, z = batch group.
template <int NB, bool PAIR>
__global__ void __launch_bounds__(kTcRings, 1) theta_inverse_tc_kernel(InvArgs a, int ntiles) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int L = a.L;
  const int rank = a.rank0 + (int)(blockIdx.x / ntiles), tile = blockIdx.x % ntiles;
  const int m = a.mpos ? rank : m_of_rank(rank);
  const int ni = PAIR ? (a.nN - 1) / 2 + (int)blockIdx.y : (int)blockIdx.y;
  const int n = ni - (a.nN - 1) / 2;
  if (PAIR && n == 0 && m < 0) return;
  const int l0 = a.seed[(size_t)ni * (2 * L - 1) + m + L - 1].l0;
  if (l0 >= L) {                 // no degree of this order: its ring values are 0
    constexpr int NBX = PAIR ? 2 * NB : NB;
    const int t = a.ring0 + tile * kTcRings + (int)threadIdx.x;
    if (t >= a.nring) return;
    for (int b = 0; b < NBX; ++b) {
      const Slot sl = slot_of<NB, PAIR>(b, blockIdx.z * NB, a.nsig, a.nN, ni, m, n, L);
      if (sl.sig_off < 0) continue;
      const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
      reinterpret_cast<double2*>(a.out)[(size_t)sl.sig_off * a.s_sig + t * a.s_t + col * a.s_m] =
          make_double2(0.0, 0.0);
    }
    return;
  }
  const int t_lo = a.ring0 + tile * kTcRings, t_hi = min(a.nring, t_lo + kTcRings) - 1;
  const bool diff = a.ring[t_lo].diff || a.ring[t_hi].diff;
  if (diff) tc_inverse_body<NB, PAIR, true>(a, m, ni, n, tile, l0, smem);
  else tc_inverse_body<NB, PAIR, false>(a, m, ni, n, tile, l0, smem);
}

template <int NB, bool PAIR>
cudaError_t launch_inv_tc(const InvArgs& a, cudaStream_t st) {
  constexpr int C = 2 * (PAIR ? 2 * NB : NB);
  const int ntiles = (a.nring - a.ring0 + kTcRings - 1) / kTcRings;
  if (ntiles == 0) return cudaSuccess;
  // at least 76 KiB per CTA, so that at most two CTAs (2 x 256 TMEM columns) share an SM
  const size_t smem = TcSmem<C>::bytes > 78 * 1024 ? TcSmem<C>::bytes : 78 * 1024;
  auto kern = theta_inverse_tc_kernel<NB, PAIR>;
  cudaError_t e = set_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nrank * ntiles, PAIR ? (a.nN + 1) / 2 : a.nN, (a.nsig + NB - 1) / NB);
  kern<<<grid, kTcRings, smem, st>>>(a, ntiles);
  return launched();
}

}  // namespace

cudaError_t launch_theta_inverse_tc(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (paired_plan(p)) {
    if (a.nsig >= 2) return launch_inv_tc<2, true>(a, st);
    return launch_inv_tc<1, true>(a, st);
  }
  if (a.nsig >= 4) return launch_inv_tc<4, false>(a, st);
  if (a.nsig >= 2) return launch_inv_tc<2, false>(a, st);
  return launch_inv_tc<1, false>(a, st);
}

int device_status(int device, bool clear, int* status) {
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return S2GB_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return S2GB_EINVAL;
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_s2gb_device_status, sizeof(int));
  if (e == cudaSuccess && clear && v != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_s2gb_device_status, &zero, sizeof(int));
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) return S2GB_ECUDA;
  *status = v;
  return S2GB_OK;
}

}  // namespace s2gb

extern "C" int s2gb_device_status(int device, int clear) {
  int v = 0;
  const int rc = s2gb::device_status(device, clear != 0, &v);
  return rc != S2GB_OK ? rc : v;
}
