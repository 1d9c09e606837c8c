// Inverse theta stage (Sec. 4.1, Eq. disc_ish_expanded; interleaved as in Sec. 4.4) with the
// contraction over the degree on the tensor cores.
//
// For one order m the stage is a product: out[t][c] = sum_l x_l(theta_t) h'_l[c], the ring x degree
// matrix of d-functions (generated on the fly by the float64 recursion of theta_kernels.cu, one
// chain per thread) times a degree x column block of coefficients (c = real and imaginary part of
// each signal slot).  On GB300 the float64 pipe (2 lanes per SM and clock) is the scarce unit: the
// recursion needs 2 of its FMAs per element, a float64 contraction 2 more per element and signal.
// Here the recursion alone stays on the float64 pipe; the contraction runs as exact integer
// arithmetic on the float16 tensor cores, after the splitting of the Ozaki scheme (Ozaki, Ogita,
// Oishi, Rump, Numer. Algorithms 59, 2012; on float16 tensor cores: Mukunoki, Ozaki, Ogita,
// Imamura, 2020):
//
//   * every recursion value becomes a fixed-point integer qa = round(x 2^(55 - rho_l)), with rho_l a
//     power-of-two bound of |x| at degree l (|u^l| <= 1/gamma_l for the normalised values,
//     |d| <= 1 in the difference form), and every coefficient qh = round(h' 2^(55 - eps_c)) with one
//     exponent eps_c per column (a bound over the degrees of the CTA's order); the scale 2^rho_l
//     moves into the coefficient of degree l, so the product is unchanged;
//   * |q| <= 2^54 is written in 7 balanced base-256 digits in [-128, 127] (adding 0x80 to every
//     byte of the two's complement integer and subtracting it again digit by digit), each digit
//     exact in float16;
//   * one tcgen05.mma per digit i of the d-values multiplies the i-th digit matrix (128 rings x
//     16 degrees) by the digits j = 0 .. 6 - i of the coefficients and accumulates the product of
//     digits (i, j) into the Tensor Memory columns of level s = i + j: the B operand holds digit j
//     in rows 16 j .. 16 j + 15 and the accumulator of MMA i starts at column 16 i.  Every digit
//     product is an integer below 2^14 in magnitude and a level receives at most 7 of them per
//     degree, so 128 degrees sum exactly below 2^24 in float32;
//   * every 128 degrees (and at the end) each thread reads its ring's 7 levels back, converts them
//     to integers and adds the weights 256^(12 - s) exactly in two 64-bit integers per column;
//     one float64 conversion at the end gives the result.  Levels s > 6 are never formed: their
//     weight is below 2^-48 of the leading ones, under the rounding of the float64 recursion.
//
// Mapping: CTA = (order rank, tile of 128 rings, n, batch group); thread tid = ring = TMEM lane; a
// tile holds 64 rings counted from the first ring and the 64 mirrored ones counted from the last,
// so that the polar caps, which need the difference form, share the first tiles.
// Per chunk of 16 degrees each thread advances its chain 16 steps, writing its 7 digit rows into
// shared memory (K-major 8 x 16-byte core matrices); 16 x slots threads write the coefficient
// digits; after a CTA barrier one thread issues the 7 MMAs and commits them to an mbarrier.  The
// operand buffers are single: the next chunk's first digits are stored only after that mbarrier
// completes, which the 8 recursion steps before the store cover.  Four CTAs share an SM (128 TMEM
// columns, 128 registers per thread, about 36 KiB of shared memory each).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "tc_common.cuh"
#include "theta_common.cuh"
#include "theta_f32.cuh"

// Status of the tensor-core kernels on this device: 0, or the first tc::kStatus* code recorded by a
// kernel whose bounded wait ran out (read and cleared by s2gb_device_status).
__device__ int g_s2gb_device_status;

namespace s2gb {

namespace {
using namespace theta;

constexpr int kTcRings = 128;        // rings per CTA = MMA M = TMEM lanes
constexpr int kTcK = 16;             // degrees per chunk = MMA K (float16)
constexpr int kDigits = 7;           // balanced base-256 digits per operand
constexpr int kLevelCols = 16;       // TMEM columns (and B rows) per digit level: up to 8 used
constexpr int kTmemCols = 128;       // 7 levels of 16 columns, allocated as 128
constexpr int kDrainChunks = 8;      // 128 degrees: 7 * 128 * 2^14 < 2^24
constexpr int kATileBytes = kTcRings * kTcK * 2;                 // one digit matrix (4 KiB)
constexpr int kABytes = kDigits * kATileBytes;                   // 28 KiB
constexpr int kBBytes = kDigits * kLevelCols * kTcK * 2;         // 3.5 KiB
constexpr int kCsOff = kABytes + kBBytes;                        // recursion coefficients [2][16][10]
constexpr int kWOff = kCsOff + 2 * kTcK * kCoefPerStepN * 8;     // coefficient factors w_j [2][16]
constexpr int kBarOff = kWOff + 2 * kTcK * 8;
constexpr int kMiscOff = kBarOff + 8;
constexpr int kSmemBytes = kMiscOff + 64;
// requested per CTA: at most four CTAs (4 x 128 TMEM columns) on an SM's 228 KiB
constexpr int kSmemRequest = 47 * 1024;

// Byte offset of element (row, k) in a K-major operand tile of 16 columns: 8-row x 16-byte core
// matrices, the two K halves 128 bytes apart (LBO), row groups 256 bytes apart (SBO).
__device__ __forceinline__ int kmajor_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// round(|x| 2^(55 - rho)) with the sign of x, plus 0x0080808080808080: byte p (p = 0..6) of the
// result is the balanced base-256 digit of weight 256^p, offset by 128.  Needs |x| < 2^(rho - 1).
// Rounding to nearest (not truncation) keeps the split unbiased, so that the errors of a sum of
// many split values do not add up in one direction.  Zero and subnormal x give the digits of 0.
__device__ __forceinline__ uint2 offset_digits(double x, int rho) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int ex = (int)((hi >> 20) & 0x7ffu);
  const uint32_t sh = ex == 0 ? 64u : (uint32_t)(1023 + rho - ex);   // >= 2 when |x| < 2^(rho-1)
  const uint64_t m = ((((uint64_t)((hi & 0xfffffu) | 0x100000u)) << 32) | lo) << 3;   // 56 bits
  uint64_t q;
  asm("shr.b64 %0, %1, %2;" : "=l"(q) : "l"(m), "r"(sh - 1));         // one fraction bit kept
  q = (q + 1) >> 1;
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

// Ring of thread `tid` in inverse tile `tile`, or -1: threads 0..63 take the tile's rings counted
// from the first ring of the launch, threads 64..127 the mirrored rings counted from the last, so
// that both polar caps (the difference form) fall into the first tiles.
__device__ __forceinline__ int inv_ring(const InvArgs& a, int tile, int tid) {
  constexpr int H = kTcRings / 2;
  const int nr = a.nring - a.ring0, half = (nr + 1) / 2;
  const int q = tile * H + (tid & (H - 1));
  if (tid < H) return q < half ? a.ring0 + q : -1;
  return q < nr - half ? a.nring - 1 - q : -1;
}

// Per-degree factor of the coefficients: w_j = scale_j (* gamma_j for normalised chains)
// * 2^rho_j, so that h'_{j,c} = h_{j,c} * sign_slot * w_j and x_j h_j = (x_j 2^-rho_j) h'_j.
template <bool DIFF>
__device__ __forceinline__ double coef_factor(const double* coef_m, const double* scale, int j) {
  const double* c = coef_m + (size_t)j * kCoefPerStepN;
  const int rho = DIFF ? 2 : exp_of(c[9]) + 2;
  return (DIFF ? scale[j] : scale[j] * c[3]) * pow2i(rho);
}

// Coefficient h_{j,b} of signal slot b (times the slot's sign), both parts; zero when inactive.
template <int NB, bool PAIR>
__device__ __forceinline__ double2 coef_raw(const InvArgs& a, int j, int b, int sig0, int ni, int m, int n, int L) {
  const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
  double2 h = make_double2(0.0, 0.0);
  if (sl.sig_off >= 0) {
    h = reinterpret_cast<const double2*>(a.flm)[((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0];
    if (a.mpos && m == 0) h.y = 0.0;
    if (sl.sign < 0) { h.x = -h.x; h.y = -h.y; }
  }
  return h;
}

template <int NB, bool PAIR, bool DIFF>
__device__ __forceinline__ void tc_inverse_body(const InvArgs& a, int m, int ni, int n, int tile, int l0,
                                                unsigned char* smem) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  constexpr int C = 2 * NBX;
  static_assert(C <= 8, "at most 8 columns per level");
  const int L = a.L, T = 2 * L - 1;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mi = m + L - 1;
  const int sig0 = blockIdx.z * NB;

  unsigned char* sA = smem;
  unsigned char* sB = smem + kABytes;
  double* cs = reinterpret_cast<double*>(smem + kCsOff);
  double* ws = reinterpret_cast<double*>(smem + kWOff);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBarOff);
  int* eps_s = reinterpret_cast<int*>(smem + kMiscOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(eps_s + 8);
  int* abort_s = reinterpret_cast<int*>(eps_s + 9);
  const uint32_t bar_a = tc::smem_addr(bar);

  const double* coef_m = a.coef + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStepN;
  const double* scale = a.scale + (size_t)ni * L;

  // ---- set-up: barrier, Tensor Memory, zero B rows, column exponent bounds, first coefficients
  if (tid == 0) {
    tc::mbar_init(bar_a, 1);
    tc::mbar_init_fence();
    *abort_s = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_slot), kTmemCols);
  for (int q = tid; q < kBBytes / 16; q += kTcRings) reinterpret_cast<uint4*>(sB)[q] = make_uint4(0, 0, 0, 0);
  if (tid < 8) eps_s[tid] = -100000;
  for (int q = tid; q < kTcK * kCoefPerStepN; q += kTcRings) {
    const int j = l0 + q / kCoefPerStepN;
    cs[q] = (j < L) ? coef_m[(size_t)l0 * kCoefPerStepN + q] : 0.0;
  }
  if (tid < kTcK) ws[tid] = (l0 + tid < L) ? coef_factor<DIFF>(coef_m, scale, l0 + tid) : 0.0;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  // |h_{j,c} w_j| < 2^(e_h + 1) 2^(e_w + 1): eps_c = max_j (e_h + e_w) + 3 bounds the column
  const int ndeg = L - l0;
  {
    int emax[C];
#pragma unroll
    for (int c = 0; c < C; ++c) emax[c] = -100000;
    for (int j = l0 + tid; j < L; j += kTcRings) {
      const int ew = exp_of(coef_factor<DIFF>(coef_m, scale, j));
#pragma unroll
      for (int b = 0; b < NBX; ++b) {
        const double2 h = coef_raw<NB, PAIR>(a, j, b, sig0, ni, m, n, L);
        if (h.x != 0.0) emax[2 * b] = max(emax[2 * b], exp_of(h.x) + ew);
        if (h.y != 0.0) emax[2 * b + 1] = max(emax[2 * b + 1], exp_of(h.y) + ew);
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int e = __reduce_max_sync(0xffffffffu, emax[c]);
      if ((tid & 31) == 0) atomicMax(&eps_s[c], e);
    }
  }
  __syncthreads();
  auto col_eps = [&](int c) { const int e = eps_s[c]; return (e < -4000 ? 0 : e) + 3; };

  // ---- the chain of this thread's ring
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  const int t = inv_ring(a, tile, tid);
  double x = 0.0, y = 0.0, v = 0.0;
  int E = 0;
  bool north = true;
  if (t >= 0) {
    const RingData rd = a.ring[t];
    seed_value(sd, rd, x, E);
    v = rd.v;
    north = rd.north;
  }
  const unsigned nmask = north ? 0x80000000u : 0u;

  // level sums, exactly: X_c = sum 2^24 L0 + 2^16 L1 + 2^8 L2 + L3, Y_c = 2^16 L4 + 2^8 L5 + L6
  long long X[C], Y[C];
#pragma unroll
  for (int c = 0; c < C; ++c) { X[c] = 0; Y[c] = 0; }

  const int nchunks = (ndeg + kTcK - 1) / kTcK;
  int since_reset = 0;
  bool ok = true;
  const uint32_t sA_addr = tc::smem_addr(sA), sB_addr = tc::smem_addr(sB);
  const int hb = tid % NBX, hj = tid / NBX;   // coefficient slot and chunk degree of this thread
  for (int k = 0; k < nchunks; ++k) {
    const int jc = l0 + k * kTcK;
    const double* csk = cs + (k & 1) * kTcK * kCoefPerStepN;
    // prefetch: the next chunk's recursion coefficients and this chunk's coefficients h
    double cpre[2] = {0.0, 0.0};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int q = tid + r * kTcRings;
      if (q < kTcK * kCoefPerStepN && jc + kTcK + q / kCoefPerStepN < L)
        cpre[r] = coef_m[(size_t)(jc + kTcK) * kCoefPerStepN + q];
    }
    double wpre = 0.0;
    if (tid < kTcK && jc + kTcK + tid < L) wpre = coef_factor<DIFF>(coef_m, scale, jc + kTcK + tid);
    double2 hpre = make_double2(0.0, 0.0);
    if (tid < kTcK * NBX && jc + hj < L) hpre = coef_raw<NB, PAIR>(a, jc + hj, hb, sig0, ni, m, n, L);

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
        if (j < L - 1) stepn<DIFF>(x, y, v, nmask, north, c);
      }
      renorm(x, y, E);
      // the previous chunk's MMAs read these buffers: they must be complete before the first store
      if (g == 0 && k > 0 && !tc::mbar_wait(bar_a, (uint32_t)((k - 1) & 1))) {
        set_status(tc::kStatusMmaWait);
        *abort_s = 1;
      }
#pragma unroll
      for (int i = 0; i < kDigits; ++i) {
        const uint4 val = live ? make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]) : make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(sA + i * kATileBytes + kmajor_off(tid, g * 8)) = val;
      }
    }
    // B digits of this chunk: thread (degree hj, slot hb) writes rows 16 i + 2 hb and 16 i + 2 hb + 1
    if (tid < kTcK * NBX) {
      const double wj = ws[(k & 1) * kTcK + hj];
      const uint2 qr = offset_digits(hpre.x * wj, col_eps(2 * hb));
      const uint2 qi = offset_digits(hpre.y * wj, col_eps(2 * hb + 1));
#pragma unroll
      for (int i = 0; i < kDigits; ++i) {
        *reinterpret_cast<unsigned short*>(sB + kmajor_off(kLevelCols * i + 2 * hb, hj)) = digit_half(qr, i);
        *reinterpret_cast<unsigned short*>(sB + kmajor_off(kLevelCols * i + 2 * hb + 1, hj)) = digit_half(qi, i);
      }
    }
    // the next chunk's recursion coefficients and factors
    {
      double* csn = cs + ((k + 1) & 1) * kTcK * kCoefPerStepN;
      csn[tid] = cpre[0];
      if (tid + kTcRings < kTcK * kCoefPerStepN) csn[tid + kTcRings] = cpre[1];
      if (tid < kTcK) ws[((k + 1) & 1) * kTcK + tid] = wpre;
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (*abort_s) { ok = false; break; }
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int i = 0; i < kDigits; ++i) {
        const uint64_t ad = tc::smem_desc(sA_addr + i * kATileBytes, 128, 256);
        const uint64_t bd = tc::smem_desc(sB_addr, 128, 256);
        // MMA 0 covers every level and (re)starts the accumulation after a read-back
        tc::mma_f16(tmem + kLevelCols * i, ad, bd, tc::idesc_f16_f32(kTcRings, kLevelCols * (kDigits - i)),
                    since_reset > 0 || i > 0);
      }
      tc::mma_commit(bar_a);
    }
    ++since_reset;
    if (since_reset == kDrainChunks || k == nchunks - 1) {
      // read the 7 levels of this ring back and add them exactly into X, Y
      if (!tc::mbar_wait(bar_a, (uint32_t)(k & 1))) {
        set_status(tc::kStatusMmaWait);
        ok = false;
      }
      tc::fence_after_sync();
      if (__all_sync(0xffffffffu, ok)) {
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        int lam[kDigits][C];
#pragma unroll
        for (int s = 0; s < kDigits; ++s) {
          uint32_t r[8];
          tc::tmem_ld8(trow + (uint32_t)(kLevelCols * s), r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < C; ++c) lam[s][c] = __float2int_rn(__uint_as_float(r[c]));
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          X[c] += ((long long)lam[0][c] << 24) + ((long long)lam[1][c] << 16) + ((long long)lam[2][c] << 8) +
                  (long long)lam[3][c];
          Y[c] += ((long long)lam[4][c] << 16) + ((long long)lam[5][c] << 8) + (long long)lam[6][c];
        }
      }
      tc::fence_before_sync();
      since_reset = 0;
      if (!__syncthreads_and(ok)) { ok = false; break; }
    }
  }

  if (ok && t >= 0) {
    // value = 2^(eps_c - 110) sum_s 256^(12 - s) L_s = 2^(eps_c - 38) (X + 2^-24 Y)
#pragma unroll
    for (int b = 0; b < NBX; ++b) {
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      if (sl.sig_off < 0) continue;
      const double re = ldexp(fma((double)Y[2 * b], 0x1p-24, (double)X[2 * b]), col_eps(2 * b) - 38);
      const double im = ldexp(fma((double)Y[2 * b + 1], 0x1p-24, (double)X[2 * b + 1]), col_eps(2 * b + 1) - 38);
      const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
      reinterpret_cast<double2*>(a.out)[(size_t)sl.sig_off * a.s_sig + t * a.s_t + col * a.s_m] =
          make_double2(re, im);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// Grid as theta_inverse_kernel: x = (rank of m) * ntiles + tile, y = n index, z = batch group.
template <int NB, bool PAIR>
__global__ void __launch_bounds__(kTcRings, 4) theta_inverse_tc_kernel(InvArgs a, int ntiles) {
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
    const int t = inv_ring(a, tile, (int)threadIdx.x);
    if (t < 0) return;
    for (int b = 0; b < NBX; ++b) {
      const Slot sl = slot_of<NB, PAIR>(b, blockIdx.z * NB, a.nsig, a.nN, ni, m, n, L);
      if (sl.sig_off < 0) continue;
      const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
      reinterpret_cast<double2*>(a.out)[(size_t)sl.sig_off * a.s_sig + t * a.s_t + col * a.s_m] =
          make_double2(0.0, 0.0);
    }
    return;
  }
  // the form of the tile: the difference form if any of its rings lies in a polar cap (the caps
  // are contiguous at both ends, so the ends of the tile's two ring ranges decide)
  const int nr = a.nring - a.ring0, half = (nr + 1) / 2;
  const int q0 = tile * (kTcRings / 2), q1 = min(half, q0 + kTcRings / 2) - 1;
  bool diff = a.ring[a.ring0 + q0].diff || a.ring[a.ring0 + q1].diff;
  if (q0 < nr - half) {
    const int r1 = min(nr - half, q0 + kTcRings / 2) - 1;
    diff = diff || a.ring[a.nring - 1 - q0].diff || a.ring[a.nring - 1 - r1].diff;
  }
  if (diff) tc_inverse_body<NB, PAIR, true>(a, m, ni, n, tile, l0, smem);
  else tc_inverse_body<NB, PAIR, false>(a, m, ni, n, tile, l0, smem);
}

template <int NB, bool PAIR>
cudaError_t launch_inv_tc(const InvArgs& a, cudaStream_t st) {
  static_assert(kSmemBytes <= kSmemRequest, "shared memory layout");
  const int ntiles = ((a.nring - a.ring0 + 1) / 2 + kTcRings / 2 - 1) / (kTcRings / 2);
  if (ntiles == 0) return cudaSuccess;
  auto kern = theta_inverse_tc_kernel<NB, PAIR>;
  cudaError_t e = set_dynamic_smem((const void*)kern, kSmemRequest);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nrank * ntiles, PAIR ? (a.nN + 1) / 2 : a.nN, (a.nsig + NB - 1) / NB);
  kern<<<grid, kTcRings, kSmemRequest, st>>>(a, ntiles);
  return launched();
}

// =============================================================================================
// Float32 inverse theta stage with the contraction on the tensor cores.  The float32 recursion of
// theta_f32.cuh (unnormalised d, |d| <= 1 once live) runs one chain per thread as in the float64
// tensor-core inverse above; the contraction is the same exact digit scheme with four balanced
// base-256 digits per operand (a float32 value to 2^-30 of its bound):
//   * q = round(d 2^29) comes from FMAs with the magic constant 1.5 2^23, whose low mantissa bits
//     hold the nearest integer: hi = round(d 2^21), then the exact remainder d 2^21 - hi (one more
//     FMA) gives lo = round(256 (d 2^21 - hi)), q = 256 hi + lo (|q| <= 2^29); the coefficients
//     h' = h scale_l become round(h' 2^(29 - eps_c)) with one exponent eps_c per column (2^eps_c
//     bounds the column);
//   * one MMA per d digit i accumulates the digit products (i, j), j <= 3 - i, into the TMEM
//     columns of level s = i + j (the dropped products of levels s > 3 amount to less than 2^-26
//     of the product of the operands' bounds, under float32 rounding; with three digits the
//     dropped level would cost about 2^-19, above it); a level receives at most 4 products of
//     magnitude <= 2^14 per degree, so 128 degrees sum exactly below 2^24 in float32;
//   * every 128 degrees each thread combines its ring's levels per column, X = 2^24 L0 + 2^16 L1 +
//     2^8 L2 + L3, in float32 (one rounding) and adds it to a float32 register sum (at most 16
//     read-backs at L = 2048); the value is X 2^(eps_c - 34).
// The level sums are exact integers, so no compensated summation is needed, and the result does
// not depend on how the signals are batched.  Up to 16 signals share one recursion (32 columns).
// =============================================================================================
constexpr int kDigits32 = 4;
constexpr int kDrain32 = 8;                // chunks of 16 degrees between read-backs: 128 degrees
constexpr float kMagic32 = 12582912.0f;    // 1.5 * 2^23

// round(256 x scale) + 0x80808080: bytes 0..3 are the balanced digits of weight 256^0..256^3,
// offset by 128.  x scale = hi + r exactly (hi the nearest integer, |r| <= 1/2, r exact in float),
// and the result is 256 hi + round(256 r).  Needs |x scale| < 2^22.
__device__ __forceinline__ uint32_t offset_digits32(float x, float scale) {
  const float y1 = fmaf(x, scale, kMagic32);
  const float hi = y1 - kMagic32;
  const float y2 = fmaf(fmaf(x, scale, -hi), 256.0f, kMagic32);
  const int q = (int)((__float_as_uint(y1) - 0x4B400000u) << 8) + (int)(__float_as_uint(y2) - 0x4B400000u);
  return (uint32_t)q + 0x80808080u;
}
// The same with scale 2^e, -108 <= e <= 145 (beyond float's 2^127 the value is scaled by 2^64
// first, exactly: it is then below 2^-100).
__device__ __forceinline__ uint32_t offset_digits32_scaled(float x, int e) {
  return e > 120 ? offset_digits32(x * 0x1p64f, pow2f(e - 64)) : offset_digits32(x, pow2f(e));
}

template <int NB>
struct InvTc32 {
  static constexpr int C = 2 * NB;                          // columns (re, im of each signal)
  static constexpr int CX = (C + 7) / 8 * 8;                // columns read back (groups of 8)
  static constexpr int LC = C <= 16 ? 16 : 32;              // TMEM columns (and B rows) per level
  static constexpr int kTmem = C <= 16 ? 64 : 128;          // 4 levels
  static constexpr int kABytes = kDigits32 * kATileBytes;   // 16 KiB
  static constexpr int kBBytes = kDigits32 * LC * kTcK * 2;
  static constexpr int kCsOff = kABytes + kBBytes;          // recursion coefficients [2][16][6]
  static constexpr int kSclOff = kCsOff + 2 * kTcK * kCoefPerStep * 4;   // scale_l [2 chunks][16]
  static constexpr int kBarOff = (kSclOff + 2 * kTcK * 4 + 7) / 8 * 8;
  static constexpr int kMiscOff = kBarOff + 8;              // eps[32], tmem slot, abort
  static constexpr int kSmem = kMiscOff + 4 * 34;
};

template <int NB, bool DIFF>
__device__ __forceinline__ void tc_inverse_body_f32(const InvArgs& a, int m, int ni, int tile, int l0,
                                                    unsigned char* smem) {
  using K = InvTc32<NB>;
  constexpr int C = K::C, CX = K::CX, LC = K::LC;
  const int L = a.L, T = 2 * L - 1;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mi = m + L - 1;
  const int sig0 = blockIdx.z * NB;

  unsigned char* sA = smem;
  unsigned char* sB = smem + K::kABytes;
  float* cs = reinterpret_cast<float*>(smem + K::kCsOff);
  float* scl = reinterpret_cast<float*>(smem + K::kSclOff);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + K::kBarOff);
  int* eps_s = reinterpret_cast<int*>(smem + K::kMiscOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(eps_s + 32);
  int* abort_s = eps_s + 33;
  const uint32_t bar_a = tc::smem_addr(bar);

  const float* coef_m = a.coef32 + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStep;
  const double* scale = a.scale + (size_t)ni * L;
  auto coef_h = [&](int j, int b) {       // h_{j,b} (times scale_j later), both parts; zero when inactive
    float2 h = make_float2(0.f, 0.f);
    const int sig = sig0 + b;
    if (sig < a.nsig) {
      h = reinterpret_cast<const float2*>(a.flm)[((size_t)(sig * a.nN + ni) * L + j) * a.flm_ld + m + a.flm_c0];
      if (a.mpos && m == 0) h.y = 0.f;
    }
    return h;
  };

  // ---- set-up: barrier, Tensor Memory, zero B rows, column exponents, first coefficients
  if (tid == 0) {
    tc::mbar_init(bar_a, 1);
    tc::mbar_init_fence();
    *abort_s = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_slot), K::kTmem);
  for (int q = tid; q < K::kBBytes / 16; q += kTcRings) reinterpret_cast<uint4*>(sB)[q] = make_uint4(0, 0, 0, 0);
  if (tid < 32) eps_s[tid] = -100000;
  for (int q = tid; q < kTcK * kCoefPerStep; q += kTcRings) {
    const int j = l0 + q / kCoefPerStep;
    cs[q] = (j < L) ? coef_m[(size_t)l0 * kCoefPerStep + q] : 0.0f;
  }
  if (tid < kTcK) scl[tid] = l0 + tid < L ? (float)scale[l0 + tid] : 0.f;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  {
    int emax[C];
#pragma unroll
    for (int c = 0; c < C; ++c) emax[c] = -100000;
    // |h scale_j| < 2^(e_h + 1) 2^(e_s + 1): the exponents added on the integer pipe
    for (int j = l0 + tid; j < L; j += kTcRings) {
      const int es = exp_of(scale[j]) + 1;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const float2 h = coef_h(j, b);
        if (h.x != 0.f) emax[2 * b] = max(emax[2 * b], expf_of(h.x) + es);
        if (h.y != 0.f) emax[2 * b + 1] = max(emax[2 * b + 1], expf_of(h.y) + es);
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int e = __reduce_max_sync(0xffffffffu, emax[c]);
      if ((tid & 31) == 0) atomicMax(&eps_s[c], e);
    }
  }
  __syncthreads();
  // |h'| < 2^eps_c (|round(h' 2^(29 - eps_c))| < 2^29); a column of zeros takes eps_c = 1
  auto col_eps = [&](int c) { const int e = eps_s[c]; return (e < -1000 ? 0 : e) + 1; };

  // ---- the chain of this thread's ring
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  const int t = inv_ring(a, tile, tid);
  float x = 0.f, y = 0.f, v = 0.f;
  int E = 0;
  bool north = true;
  if (t >= 0) {
    const RingData rd = a.ring[t];
    seed_value_f32(sd, rd, x, E);
    v = a.v32[t];
    north = rd.north;
  }
  if (DIFF) y = x;
  const unsigned nmask = north ? 0x80000000u : 0u;
  // a chain that is live (|d| >= 2^-90) stays live: once the whole warp is, the bookkeeping stops
  bool all_live = __all_sync(0xffffffffu, E == 0);
  bool live = __any_sync(0xffffffffu, E == 0);

  float X[CX];
#pragma unroll
  for (int c = 0; c < CX; ++c) X[c] = 0.f;

  const int nchunks = (L - l0 + kTcK - 1) / kTcK;
  int since_reset = 0;
  bool ok = true;
  const uint32_t sA_addr = tc::smem_addr(sA), sB_addr = tc::smem_addr(sB);
  for (int k = 0; k < nchunks; ++k) {
    const int jc = l0 + k * kTcK;
    const float* csk = cs + (k & 1) * kTcK * kCoefPerStep;
    // prefetch: the next chunk's recursion coefficients and scales, this chunk's coefficients h
    float cpre = 0.f;
    if (tid < kTcK * kCoefPerStep && jc + kTcK + tid / kCoefPerStep < L)
      cpre = coef_m[(size_t)(jc + kTcK) * kCoefPerStep + tid];
    float spre = 0.f;
    if (tid < kTcK && jc + kTcK + tid < L) spre = (float)scale[jc + kTcK + tid];
    constexpr int kHPer = (kTcK * NB + kTcRings - 1) / kTcRings;      // entries per thread
    float2 hpre[kHPer];
#pragma unroll
    for (int r = 0; r < kHPer; ++r) {
      const int q = tid + r * kTcRings, hj = q / NB, hb = q % NB;
      hpre[r] = (q < kTcK * NB && jc + hj < L) ? coef_h(jc + hj, hb) : make_float2(0.f, 0.f);
    }

#pragma unroll
    for (int g = 0; g < 2; ++g) {
      // digits of the values of degrees jc + 8g .. +7, as pairs of float16 (0 for dead chains)
      uint32_t w[kDigits32][4];
      bool any = false;
      uint32_t q0 = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int jj = g * 8 + u, j = jc + jj;
        if (live) {
          const float xl = (E == 0 && j < L) ? x : 0.f;
          const uint32_t q = offset_digits32(xl, 2097152.0f);          // 2^21: q ~ d 2^29
          if (u & 1) {
            w[0][u >> 1] = digit_pair(q0, q, 3);
            w[1][u >> 1] = digit_pair(q0, q, 2);
            w[2][u >> 1] = digit_pair(q0, q, 1);
            w[3][u >> 1] = digit_pair(q0, q, 0);
          } else {
            q0 = q;
          }
        } else if (u & 1) {
          w[0][u >> 1] = 0u;
          w[1][u >> 1] = 0u;
          w[2][u >> 1] = 0u;
          w[3][u >> 1] = 0u;
        }
        any = any || live;
        if (j < L - 1) {
          const float* cp = csk + jj * kCoefPerStep;
          const StepCoef32 c = {cp[0], cp[1], cp[2], cp[3], cp[4], cp[5]};
          step_f32<DIFF>(x, y, v, nmask, north, c);
        }
        if ((u & 1) && !all_live) {     // every 2 steps: float32's range (kRescale32)
          renorm_f32(x, y, E);
          all_live = __all_sync(0xffffffffu, E == 0);
          live = __any_sync(0xffffffffu, E == 0);
        }
      }
      // the previous chunk's MMAs read these buffers: they must be complete before the first store
      if (g == 0 && k > 0 && !tc::mbar_wait(bar_a, (uint32_t)((k - 1) & 1))) {
        set_status(tc::kStatusMmaWait);
        *abort_s = 1;
      }
#pragma unroll
      for (int i = 0; i < kDigits32; ++i) {
        const uint4 val = any ? make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]) : make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(sA + i * kATileBytes + kmajor_off(tid, g * 8)) = val;
      }
    }
    // B digits of this chunk: entry (degree hj, signal hb) gives rows LC i + 2 hb and LC i + 2 hb + 1
#pragma unroll
    for (int r = 0; r < kHPer; ++r) {
      const int q = tid + r * kTcRings, hj = q / NB, hb = q % NB;
      if (q >= kTcK * NB) break;
      const float sj = scl[(k & 1) * kTcK + hj];
      const float2 h = make_float2(hpre[r].x * sj, hpre[r].y * sj);
      const uint32_t qr = offset_digits32_scaled(h.x, 21 - col_eps(2 * hb));
      const uint32_t qi = offset_digits32_scaled(h.y, 21 - col_eps(2 * hb + 1));
#pragma unroll
      for (int i = 0; i < kDigits32; ++i) {
        const int p = 3 - i;
        const float dr = (float)((int)((qr >> (8 * p)) & 0xffu) - 128);
        const float di = (float)((int)((qi >> (8 * p)) & 0xffu) - 128);
        *reinterpret_cast<__half*>(sB + kmajor_off(LC * i + 2 * hb, hj)) = __float2half_rn(dr);
        *reinterpret_cast<__half*>(sB + kmajor_off(LC * i + 2 * hb + 1, hj)) = __float2half_rn(di);
      }
    }
    if (tid < kTcK * kCoefPerStep) cs[((k + 1) & 1) * kTcK * kCoefPerStep + tid] = cpre;
    if (tid < kTcK) scl[((k + 1) & 1) * kTcK + tid] = spre;
    tc::fence_proxy_async();
    __syncthreads();
    if (*abort_s) { ok = false; break; }
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int i = 0; i < kDigits32; ++i) {
        const uint64_t ad = tc::smem_desc(sA_addr + i * kATileBytes, 128, 256);
        const uint64_t bd = tc::smem_desc(sB_addr, 128, 256);
        tc::mma_f16(tmem + LC * i, ad, bd, tc::idesc_f16_f32(kTcRings, LC * (kDigits32 - i)),
                    since_reset > 0 || i > 0);
      }
      tc::mma_commit(bar_a);
    }
    ++since_reset;
    if (since_reset == kDrain32 || k == nchunks - 1) {
      if (!tc::mbar_wait(bar_a, (uint32_t)(k & 1))) {
        set_status(tc::kStatusMmaWait);
        ok = false;
      }
      tc::fence_after_sync();
      if (__all_sync(0xffffffffu, ok)) {
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int h8 = 0; h8 < CX / 8; ++h8) {
          uint32_t r[kDigits32][8];
#pragma unroll
          for (int s = 0; s < kDigits32; ++s) tc::tmem_ld8(trow + (uint32_t)(LC * s + 8 * h8), r[s]);
          tc::tmem_ld_wait();
          // the levels are exact integers in float32: 2^24 L0 + 2^16 L1 + 2^8 L2 + L3, one rounding
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float v3 = fmaf(__uint_as_float(r[2][e]), 256.f, __uint_as_float(r[3][e]));
            const float v = fmaf(fmaf(__uint_as_float(r[0][e]), 256.f, __uint_as_float(r[1][e])), 65536.f, v3);
            X[8 * h8 + e] += v;
          }
        }
      }
      tc::fence_before_sync();
      since_reset = 0;
      if (!__syncthreads_and(ok)) { ok = false; break; }
    }
  }

  if (ok && t >= 0) {
    const long long col = a.m_mod ? (m >= 0 ? m : m + a.mmod) : mi;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int sig = sig0 + b;
      if (sig >= a.nsig) continue;
      const int er = col_eps(2 * b) - 34, ei = col_eps(2 * b + 1) - 34;
      const float re = (X[2 * b] * pow2f(er / 2)) * pow2f(er - er / 2);
      const float im = (X[2 * b + 1] * pow2f(ei / 2)) * pow2f(ei - ei / 2);
      reinterpret_cast<float2*>(a.out)[(size_t)(sig * a.nN + ni) * a.s_sig + t * a.s_t + col * a.s_m] =
          make_float2(re, im);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, K::kTmem);
  }
}

// Grid as the float64 tensor-core inverse: x = (rank of m) * ntiles + tile, y = n index, z =
// batch group of NB signals.
template <int NB>
__global__ void __launch_bounds__(kTcRings, 4) theta_inverse_tc_kernel_f32(InvArgs a, int ntiles) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int L = a.L;
  const int rank = a.rank0 + (int)(blockIdx.x / ntiles), tile = blockIdx.x % ntiles;
  const int m = a.mpos ? rank : m_of_rank(rank);
  const int ni = (int)blockIdx.y;
  const int l0 = a.seed[(size_t)ni * (2 * L - 1) + m + L - 1].l0;
  if (l0 >= L) {                 // no degree of this order: its ring values are 0
    const int t = inv_ring(a, tile, (int)threadIdx.x);
    if (t < 0) return;
    const long long col = a.m_mod ? (m >= 0 ? m : m + a.mmod) : m + L - 1;
    for (int b = 0; b < NB; ++b) {
      const int sig = blockIdx.z * NB + b;
      if (sig < a.nsig)
        reinterpret_cast<float2*>(a.out)[(size_t)(sig * a.nN + ni) * a.s_sig + t * a.s_t + col * a.s_m] =
            make_float2(0.f, 0.f);
    }
    return;
  }
  const int nr = a.nring - a.ring0, half = (nr + 1) / 2;
  const int q0 = tile * (kTcRings / 2), q1 = min(half, q0 + kTcRings / 2) - 1;
  bool diff = a.ring[a.ring0 + q0].diff || a.ring[a.ring0 + q1].diff;
  if (q0 < nr - half) {
    const int r1 = min(nr - half, q0 + kTcRings / 2) - 1;
    diff = diff || a.ring[a.nring - 1 - q0].diff || a.ring[a.nring - 1 - r1].diff;
  }
  if (diff) tc_inverse_body_f32<NB, true>(a, m, ni, tile, l0, smem);
  else tc_inverse_body_f32<NB, false>(a, m, ni, tile, l0, smem);
}

template <int NB>
cudaError_t launch_inv_tc32(const InvArgs& a, cudaStream_t st) {
  const int ntiles = ((a.nring - a.ring0 + 1) / 2 + kTcRings / 2 - 1) / (kTcRings / 2);
  if (ntiles == 0) return cudaSuccess;
  auto kern = theta_inverse_tc_kernel_f32<NB>;
  constexpr int smem = (InvTc32<NB>::kSmem + 1023) / 1024 * 1024 + 1024;
  cudaError_t e = set_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nrank * ntiles, a.nN, (a.nsig + NB - 1) / NB);
  kern<<<grid, kTcRings, smem, st>>>(a, ntiles);
  return launched();
}

// =============================================================================================
// Forward theta stage (Sec. 4.1, Eq. disc_sh_expanded) with the contraction over the rings on the
// tensor cores: flm[l][c] = scale_l sum_t d^l(theta_t) g'_t[c], g' the ring data times the ring
// weight and the slot sign.  The sum runs over the rings, across the threads of a CTA (one chain,
// i.e. one ring, per thread: 256 threads and 256 rings per CTA) and across the CTAs of the order.
//
//   * The ring data are split once per CTA into 7 digits per column (B operand: columns 8 j + c,
//     N = 64 with the zero digit 7; K = 256 rings, K-major), with one exponent per column over all
//     rings of the order, agreed by the CTAs through distributed shared memory.
//   * Per chunk of 16 degrees the recursion values are split as in the inverse (A operand: rows
//     16 i + l = (digit i, degree l), M = 128 of which 112 are used, K = 256 rings, stored
//     N-major: each thread writes 16-byte rows of 8 degrees) and 16 MMAs (16 rings each) form
//     every digit product S_ij(c, l) in Tensor Memory.  A tile sums at most 256 rings: |S_ij| <=
//     2^22, exact in float32.
//   * Each accumulator row (i, l) folds its products into two exact 64-bit words per column,
//     X = sum_{i+j<=3} 256^(3-i-j) S_ij and Y = sum_{4<=i+j<=6} 256^(6-i-j) S_ij.  The rows of
//     digits 2q and 2q + 1 lie in TMEM lane quadrant q, which warps q and q + 4 share: they read
//     back complementary ranges of the coefficient digits j <= 6 - 2q.  Each warp adds its two
//     digit rows of a degree with one shuffle; the warps' words of a degree are added through
//     shared memory, and the tiles of the order through distributed shared memory of the
//     thread-block cluster (one cluster per order, up to 8 tiles), in integers: the result does
//     not depend on the order of the additions.
//   * Every tile gets an equal share of the polar-cap rings, which run the difference form, in
//     its last warps (the same number in every tile), and of the other rings in the rest, so the
//     CTAs of a cluster do the same work and none paces the others at the cluster barriers.  The
//     difference form carries d itself; its values are scaled by 1 / gamma_l before the split, so
//     that every ring's digits share the scale of the normalised values u = d / gamma_l and one
//     accumulator serves both forms.
//   * The loop is software-pipelined: a chunk's accumulator is read back in the middle of the next
//     chunk's recursion, and the cluster's sums of chunk k are formed during chunk k + 2.
//   * Two CTAs (16 warps) share an SM: 110 KiB of shared memory and at most 128 registers per
//     thread each.
// =============================================================================================
constexpr int kFwdN = kDigits * kTcK;             // 112 = (d digit i, degree l)
constexpr int kFwdM = 64;                         // 8 j + c: coefficient digit j, column c (MMA N)
constexpr int kFwdThreads = 2 * kTcRings;         // one ring per thread
constexpr int kFwdRings = kFwdThreads;            // rings per CTA
constexpr int kFwdWarps = kFwdThreads / 32;
constexpr int kFwdMaxTiles = 8;                   // 2048 rings per order
constexpr int kFwdTmemCols = 64;
constexpr int kGBytes = kFwdM * kFwdRings * 2;    // 32 KiB
constexpr int kDBytes = kFwdRings * kFwdN * 2;    // 56 KiB
constexpr int kFwdStageOff = kGBytes + kDBytes;                       // [8 warps][8 c][16 l] x (X, Y)
constexpr int kFwdClOff = kFwdStageOff + kFwdWarps * 8 * kTcK * 16;   // [2 buf][8 c][16 l] x (X, Y)
constexpr int kFwdCsOff = kFwdClOff + 2 * 8 * kTcK * 16;
constexpr int kFwdFuOff = kFwdCsOff + 2 * kTcK * kCoefPerStepN * 8;   // [4 chunks][16 l] output factors
constexpr int kFwdBarOff = kFwdFuOff + 4 * kTcK * 8;
constexpr int kFwdMiscOff = kFwdBarOff + 8;       // eps_loc[8], tmem_slot, abort
constexpr int kFwdSmemBytes = kFwdMiscOff + 64;
constexpr int kFwdSmemRequest = 112 * 1024;       // two CTAs per SM
static_assert(kTcK * kCoefPerStepN + kTcK <= kFwdThreads, "one coefficient prefetch per thread");

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t peer_addr(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ long long ld_peer_s64(uint32_t addr) {
  long long v;
  asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int ld_peer_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Byte offset of (row r, ring k) in the coefficient-digit tile: K-major, 256 rings per row.
__device__ __forceinline__ int gtile_off(int r, int k) {
  return (r >> 3) * (kFwdRings / 8 * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// Byte offset of (ring k, n / 8 = 2 i + degree half) in the d-digit tile: N-major 16-byte rows.
__device__ __forceinline__ int dtile_off(int k, int n8) {
  return (k >> 3) * (kFwdN / 8) * 128 + n8 * 128 + (k & 7) * 16;
}

// Exact integer of a float32 holding an integer of magnitude below 2^22.
__device__ __forceinline__ int small_int(uint32_t bits) {
  return (int)(__float_as_uint(__uint_as_float(bits) + 12582912.0f) - 0x4B400000u);
}

// Eight recursion steps of one chain from degree j0 (cs8: the coefficients of those steps), the
// digits of the eight values it passes (0 when the chain is dead or past L) packed into w as the
// d-digit tile stores them.  DF: the difference form, whose values d are scaled by 1 / gamma_l to
// the scale of the normalised values u = d / gamma_l before the split.
template <bool DF>
__device__ __forceinline__ void fwd_steps8(double& x, double& y, double v, unsigned nmask, bool north, int E,
                                           bool live, const double* cs8, int j0, int L,
                                           uint32_t (&w)[kDigits][4]) {
  uint2 q0 = make_uint2(0, 0);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int j = j0 + u;
    const StepN c = stepn_at(cs8 + u * kCoefPerStepN);
    if (live) {
      const double xl = (E == 0 && j < L) ? (DF ? x * c.ig : x) : 0.0;
      const uint2 q = offset_digits(xl, exp_of(c.ig) + 2);
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
    if (j < L - 1) stepn<DF>(x, y, v, nmask, north, c);
  }
}

template <int NB, bool PAIR>
__device__ __forceinline__ void tc_forward_body(const FwdArgs& a, int m, int ni, int n, int tile, int ntiles,
                                                int l0, unsigned char* smem) {
  constexpr int NBX = PAIR ? 2 * NB : NB;
  constexpr int C = 2 * NBX;
  static_assert(C <= 8, "at most 8 columns");
  const int L = a.L, T = 2 * L - 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mi = m + L - 1;
  const int sig0 = blockIdx.z * NB;
  const uint32_t crank = cluster_rank();

  unsigned char* sG = smem;
  unsigned char* sD = smem + kGBytes;
  longlong2* stage = reinterpret_cast<longlong2*>(smem + kFwdStageOff);
  longlong2* cl = reinterpret_cast<longlong2*>(smem + kFwdClOff);
  double* cs = reinterpret_cast<double*>(smem + kFwdCsOff);
  double* fu = reinterpret_cast<double*>(smem + kFwdFuOff);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kFwdBarOff);
  int* eps_loc = reinterpret_cast<int*>(smem + kFwdMiscOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(eps_loc + 8);
  int* abort_s = eps_loc + 9;
  const uint32_t bar_a = tc::smem_addr(bar);
  double2* const outb = reinterpret_cast<double2*>(a.flm);

  const double* coef_m = a.coef + ((size_t)ni * T + mi) * (size_t)L * kCoefPerStepN;
  const double* scale = a.scale + (size_t)ni * L;
  // The launch's rings: ncn polar-cap rings at the front, ncs at the back (contiguous: sin theta
  // is monotone on each half), the plain rings between them.  The last wd warps of every tile run
  // the difference form on the caps, 32 wd rings per tile (then on the plain rings that the plain
  // slots of all tiles cannot hold); the other warps run the plain rings.  The last warps have the
  // least read-back work (lane quadrant 3 needs one load, taken by warp 3), which balances the
  // difference form's extra float64 instructions.
  int ncn = 0, ncs = 0;
  {
    const int half = (a.nrows + 1) / 2;
    for (int t0 = 0; t0 < a.nrows; t0 += kFwdThreads) {
      const int t = t0 + tid;
      const bool cap = t < a.nrows && a.ring[a.row0 + t].diff;
      ncn += __syncthreads_count(cap && t < half);
      ncs += __syncthreads_count(cap && t >= half);
    }
  }
  const int ncap = ncn + ncs;
  const int wd = (ncap + 32 * ntiles - 1) / (32 * ntiles);          // difference-form warps per tile
  const int dslots = 32 * wd, pslots = kFwdThreads - dslots;
  const int nplain = a.nrows - ncap;
  const int nplain_p = min(nplain, ntiles * pslots);                 // plain rings in plain slots
  const bool dform = warp >= kFwdWarps - wd;
  int tr = 0;
  bool tact;
  if (dform) {
    const int s = tile * dslots + (tid - pslots);
    tact = s < ncap + (nplain - nplain_p);
    tr = s < ncn ? a.row0 + s : s < ncap ? a.row0 + a.nrows - 1 - (s - ncn) : a.row0 + ncn + nplain_p + (s - ncap);
  } else {
    const int p = tile * pslots + tid;
    tact = p < nplain_p;
    tr = a.row0 + ncn + p;
  }
  // output factor of degree l of a chunk: gamma_l scale_l 2^(rho_l - 38), rho_l = exponent of
  // 1 / gamma_l + 2 (the column exponent is applied at the end)
  auto out_factor = [&](int l) {
    const double* cc = coef_m + (size_t)l * kCoefPerStepN;
    return ldexp(cc[3] * scale[l], exp_of(cc[9]) + 2 - 38);
  };

  // ---- set-up: barrier, Tensor Memory, the degrees below l0, column exponents over the cluster
  if (tid == 0) {
    tc::mbar_init(bar_a, 1);
    tc::mbar_init_fence();
    *abort_s = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_slot), kFwdTmemCols);
  for (int q = tid; q < kGBytes / 16; q += kFwdThreads) reinterpret_cast<uint4*>(sG)[q] = make_uint4(0, 0, 0, 0);
  if (tid < 8) eps_loc[tid] = -100000;
  if (tile == 0) {
    const int lz = min(l0, L);
    for (int q = tid; q < NBX * lz; q += kFwdThreads) {
      const int b = q / lz, j = q % lz;
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      if (sl.sig_off >= 0) outb[((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0] = make_double2(0.0, 0.0);
    }
  }
  if (tid < kTcK * kCoefPerStepN) {
    const int j = l0 + tid / kCoefPerStepN;
    cs[tid] = (j < L) ? coef_m[(size_t)l0 * kCoefPerStepN + tid] : 0.0;
  } else if (tid < kTcK * kCoefPerStepN + kTcK) {
    const int l = l0 + tid - kTcK * kCoefPerStepN;
    fu[tid - kTcK * kCoefPerStepN] = l < L ? out_factor(l) : 0.0;
  }
  double2 gv[NBX];
  {
    int emax[C];
#pragma unroll
    for (int c = 0; c < C; ++c) emax[c] = -100000;
#pragma unroll
    for (int b = 0; b < NBX; ++b) {
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      double2 g = make_double2(0.0, 0.0);
      if (tact && sl.sig_off >= 0) {
        const long long col = a.m_mod ? (sl.m >= 0 ? sl.m : sl.m + a.mmod) : sl.mi;
        g = reinterpret_cast<const double2*>(a.g)[(size_t)sl.sig_off * a.s_sig + tr * a.s_t + col * a.s_m];
        const double w = (a.use_nu ? a.nu[tr] : 1.0) * sl.sign;
        g.x *= w;
        g.y *= w;
      }
      gv[b] = g;
      if (g.x != 0.0) emax[2 * b] = max(emax[2 * b], exp_of(g.x));
      if (g.y != 0.0) emax[2 * b + 1] = max(emax[2 * b + 1], exp_of(g.y));
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int e = __reduce_max_sync(0xffffffffu, emax[c]);
      if (lane == 0) atomicMax(&eps_loc[c], e);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  cluster_arrive();
  cluster_wait();                            // every CTA's eps_loc and form are written
  int eps[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    int e = -100000;
    for (int q = 0; q < ntiles; ++q) e = max(e, ld_peer_s32(peer_addr(tc::smem_addr(&eps_loc[c]), (uint32_t)q)));
    eps[c] = (e < -2000 ? 0 : e) + 2;        // |g'| < 2^(eps_c - 1)
  }
  auto col_eps = [&](int c) {
    int e = eps[0];
#pragma unroll
    for (int q = 1; q < C; ++q) e = (c == q) ? eps[q] : e;
    return e;
  };

  // the B operand: digit j of column c in row 8 j + c, this thread's ring in column tid
#pragma unroll
  for (int b = 0; b < NBX; ++b) {
    const uint2 qr = offset_digits(gv[b].x, eps[2 * b]);
    const uint2 qi = offset_digits(gv[b].y, eps[2 * b + 1]);
#pragma unroll
    for (int j = 0; j < kDigits; ++j) {
      *reinterpret_cast<unsigned short*>(sG + gtile_off(8 * j + 2 * b, tid)) = digit_half(qr, j);
      *reinterpret_cast<unsigned short*>(sG + gtile_off(8 * j + 2 * b + 1, tid)) = digit_half(qi, j);
    }
  }

  // ---- the chain of this thread's ring
  const SeedData sd = a.seed[(size_t)ni * T + mi];
  double x = 0.0, y = 0.0, v = 0.0;
  int E = 0;
  bool north = true;
  if (tact) {
    const RingData rd = a.ring[tr];
    seed_value(sd, rd, x, E);
    v = rd.v;
    north = rd.north;
  }
  const unsigned nmask = north ? 0x80000000u : 0u;

  const int ndeg = L - l0;
  const int nchunks = (ndeg + kTcK - 1) / kTcK;
  const uint32_t sG_addr = tc::smem_addr(sG), sD_addr = tc::smem_addr(sD);
  const uint32_t cl_addr = tc::smem_addr(cl);
  bool ok = true;

  // sum over the cluster's tiles of chunk kk's (X, Y), per form, and write the owned coefficients
  auto reduce_chunk = [&](int kk) {
    const int buf = kk & 1;
    for (int p = tid * ntiles + (int)crank; p < C * kTcK; p += ntiles * kFwdThreads) {
      const int c = p % C, ll = p / C, l = l0 + kk * kTcK + ll;
      if (l >= L) continue;
      const int b = c >> 1;
      const Slot sl = slot_of<NB, PAIR>(b, sig0, a.nsig, a.nN, ni, m, n, L);
      if (sl.sig_off < 0) continue;
      long long Xs = 0, Ys = 0;
      const uint32_t off = cl_addr + (uint32_t)(((buf * 8 + c) * kTcK + ll) * 16);
      for (int q = 0; q < ntiles; ++q) {
        const uint32_t pa = peer_addr(off, (uint32_t)q);
        Xs += ld_peer_s64(pa);
        Ys += ld_peer_s64(pa + 8);
      }
      // the digits hold u = d / gamma_l at 2^-rho_l: times gamma_l 2^rho_l
      const double val = ldexp(fma((double)Ys, 0x1p-24, (double)Xs) * fu[(kk & 3) * kTcK + ll], col_eps(c));
      reinterpret_cast<double*>(outb + ((size_t)sl.sig_off * L + l) * a.flm_ld + sl.m + a.flm_c0)[c & 1] = val;
    }
  };

  // accumulator row 16 i + l (d digit i, degree l) is TMEM lane 32 q + lane, q = warp % 4: lane
  // quadrant q holds the digits i = 2q, 2q + 1, which need the coefficient digits j <= 6 - 2q
  // (columns 8 j + c); warp q reads j < jsplit, warp q + 4 the rest
  const int quad = warp & 3;
  const int ri = (32 * quad + lane) >> 4, rl = lane & 15;
  const int jmax = kDigits - 1 - 2 * quad;
  const int jsplit = (jmax + 2) / 2;
  const int jlo = warp < 4 ? 0 : jsplit, jhi = warp < 4 ? jsplit - 1 : jmax;
  for (int k = 0; k <= nchunks; ++k) {
    const bool comp = k < nchunks;
    const int jc = l0 + k * kTcK;
    const double* csk = cs + (k & 1) * kTcK * kCoefPerStepN;
    double cpre = 0.0;
    if (comp && tid < kTcK * kCoefPerStepN && jc + kTcK + tid / kCoefPerStepN < L)
      cpre = coef_m[(size_t)(jc + kTcK) * kCoefPerStepN + tid];
    else if (comp && tid >= kTcK * kCoefPerStepN && tid < kTcK * kCoefPerStepN + kTcK &&
             jc + kTcK + tid - kTcK * kCoefPerStepN < L)
      cpre = out_factor(jc + kTcK + tid - kTcK * kCoefPerStepN);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      uint32_t w[kDigits][4];
      bool live = false;
      if (comp) {
        live = __any_sync(0xffffffffu, E == 0);
        const double* cs8 = csk + g * 8 * kCoefPerStepN;
        if (dform) fwd_steps8<true>(x, y, v, nmask, north, E, live, cs8, jc + g * 8, L, w);
        else fwd_steps8<false>(x, y, v, nmask, north, E, live, cs8, jc + g * 8, L, w);
        renorm(x, y, E);
      }
      // chunk k-1's MMAs read the d-digit tile: they must be done before its first store
      if (g == 0 && k > 0 && ok) {
        if (!tc::mbar_wait(bar_a, (uint32_t)((k - 1) & 1))) {
          set_status(tc::kStatusMmaWait);
          *abort_s = 1;
        }
        tc::fence_after_sync();
      }
      if (comp) {
#pragma unroll
        for (int i = 0; i < kDigits; ++i) {
          const uint4 val = live ? make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]) : make_uint4(0, 0, 0, 0);
          *reinterpret_cast<uint4*>(sD + dtile_off(tid, 2 * i + g)) = val;
        }
      }
      if (g == 0 && k > 0 && ok) {
        // read chunk k-1's digit products back: this lane's d digit ri and degree rl against the
        // coefficient digits j of this warp's range (8 columns c each)
        long long Xs[8], Ys[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) { Xs[c] = 0; Ys[c] = 0; }
        for (int j = jlo; j <= jhi; ++j) {
          uint32_t r[8];
          tc::tmem_ld8(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(8 * j), r);
          tc::tmem_ld_wait();
          const int sdeg = ri + j;
          const bool inX = sdeg <= 3, inY = sdeg >= 4 && sdeg <= 6;
          const int shX = inX ? 8 * (3 - sdeg) : 0, shY = inY ? 8 * (6 - sdeg) : 0;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const long long S = (long long)small_int(r[c]);
            Xs[c] += inX ? (S << shX) : 0;
            Ys[c] += inY ? (S << shY) : 0;
          }
        }
        // the two digit rows of a degree (lanes rl and rl + 16), then one word pair per warp
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          Xs[c] += __shfl_xor_sync(0xffffffffu, Xs[c], 16);
          Ys[c] += __shfl_xor_sync(0xffffffffu, Ys[c], 16);
        }
        if (lane < kTcK) {
#pragma unroll
          for (int c = 0; c < 8; ++c) stage[(warp * 8 + c) * kTcK + rl] = make_longlong2(Xs[c], Ys[c]);
        }
        tc::fence_before_sync();
      }
    }
    if (comp && tid < kTcK * kCoefPerStepN) cs[((k + 1) & 1) * kTcK * kCoefPerStepN + tid] = cpre;
    else if (comp && tid < kTcK * kCoefPerStepN + kTcK) fu[((k + 1) & 3) * kTcK + tid - kTcK * kCoefPerStepN] = cpre;
    tc::fence_proxy_async();
    __syncthreads();
    if (*abort_s) ok = false;
    if (comp && ok && tid == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int ks = 0; ks < kFwdRings / kTcK; ++ks) {
        // A: d digits, M = 128 rows (i, l) (rows 112..127 read the next ring group's bytes and
        // are never read back), N-major; B: coefficient digits, N = 64 columns (j, c), K-major
        const uint64_t ad = tc::smem_desc(sD_addr + ks * 2 * (kFwdN / 8) * 128, (kFwdN / 8) * 128, 128);
        const uint64_t bd = tc::smem_desc(sG_addr + ks * 256, 128, kFwdRings / 8 * 128);
        tc::mma_f16(tmem, ad, bd, tc::idesc_f16_f32(kTcRings, kFwdM) | (1u << 15), ks > 0);
      }
      tc::mma_commit(bar_a);
    }
    if (k > 0) {
      // the cluster's sums of chunk k-2, then this tile's sums of chunk k-1 for the cluster
      if (k > 1) {
        cluster_wait();
        if (ok) reduce_chunk(k - 2);
      }
      if (tid < 8 * kTcK) {
        const int cc = tid / kTcK, ll = tid % kTcK;
        long long X = 0, Y = 0;
#pragma unroll
        for (int w8 = 0; w8 < kFwdWarps; ++w8) {
          const longlong2 sv = stage[(w8 * 8 + cc) * kTcK + ll];
          X += sv.x;
          Y += sv.y;
        }
        cl[(((k - 1) & 1) * 8 + cc) * kTcK + ll] = make_longlong2(X, Y);
      }
      __syncthreads();                       // the staging area is read: the next read-back may write it
      cluster_arrive();
    }
  }
  cluster_wait();
  if (ok) reduce_chunk(nchunks - 1);
  cluster_arrive();                          // peers may still read this CTA's shared memory
  cluster_wait();
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kFwdTmemCols);
  }
}

// Grid: x = (rank of m) * ntiles + tile (a cluster of ntiles CTAs per order), y = n index,
// z = batch group.
template <int NB, bool PAIR>
__global__ void __launch_bounds__(kFwdThreads, 2) theta_forward_tc_kernel(FwdArgs a, int ntiles) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int L = a.L;
  const int rank = a.rank0 + (int)(blockIdx.x / ntiles), tile = blockIdx.x % ntiles;
  const int m = a.mpos ? rank : m_of_rank(rank);
  const int ni = PAIR ? (a.nN - 1) / 2 + (int)blockIdx.y : (int)blockIdx.y;
  const int n = ni - (a.nN - 1) / 2;
  const int l0 = a.seed[(size_t)ni * (2 * L - 1) + m + L - 1].l0;
  // the whole cluster leaves together (uniform over its CTAs)
  if ((PAIR && n == 0 && m < 0)) return;
  if (l0 >= L) {
    if (tile == 0) {
      constexpr int NBX = PAIR ? 2 * NB : NB;
      for (int q = threadIdx.x; q < NBX * L; q += blockDim.x) {
        const int b = q / L, j = q % L;
        const Slot sl = slot_of<NB, PAIR>(b, blockIdx.z * NB, a.nsig, a.nN, ni, m, n, L);
        if (sl.sig_off >= 0)
          reinterpret_cast<double2*>(a.flm)[((size_t)sl.sig_off * L + j) * a.flm_ld + sl.m + a.flm_c0] =
              make_double2(0.0, 0.0);
      }
    }
    return;
  }
  tc_forward_body<NB, PAIR>(a, m, ni, n, tile, ntiles, l0, smem);
}

template <int NB, bool PAIR>
cudaError_t launch_fwd_tc(const FwdArgs& a, cudaStream_t st) {
  static_assert(kFwdSmemBytes <= kFwdSmemRequest, "shared memory layout");
  const int ntiles = (a.nrows + kFwdRings - 1) / kFwdRings;
  if (ntiles == 0) return cudaSuccess;
  if (ntiles > kFwdMaxTiles) return cudaErrorInvalidValue;
  auto kern = theta_forward_tc_kernel<NB, PAIR>;
  cudaError_t e = set_dynamic_smem((const void*)kern, kFwdSmemRequest);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.nrank * ntiles, PAIR ? (a.nN + 1) / 2 : a.nN, (a.nsig + NB - 1) / NB);
  cfg.blockDim = dim3(kFwdThreads, 1, 1);
  cfg.dynamicSmemBytes = kFwdSmemRequest;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)ntiles;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, a, ntiles);
  if (e != cudaSuccess) return e;
  return launched();
}

// =============================================================================================
// The forward's theta-direction quadrature operator on the tensor cores.
//
// For one order row the operator maps the ring values F(theta_t'), t' < R, to the values H(theta_t)
// the forward theta kernel integrates: the torus extension (Sec. 4.2.2: the reflected ring times
// sigma = (-1)^(m-n), (1 + sigma)/2 on a self-reflected ring) followed by the FFT operator of the
// quadrature (weights on a fine grid, projection to the bandlimit), restricted to the R rings.  It
// is linear, real and the same for every row of a given parity: H = Q_sigma F with two R x R real
// matrices, built at plan creation from the FFT operator's responses to unit vectors.  Applying
// them is a GEMM over the rings (K = R): rows t (128 per CTA, the A operand: Q_sigma digits copied
// per chunk of 16 rings by a TMA bulk copy from the plan's tiles), columns = 8 orders of one parity
// x (re, im) (the B operand: the spectra split into digits in the CTA), with the digit levels
// merged in Tensor Memory and read back exactly every 128 rings, as in the inverse theta stage.
// =============================================================================================
constexpr int kOpCols = 16;                                   // 8 orders x (re, im)
constexpr int kOpATile = kDigits * kTcRings * kTcK;           // fp16 elements of one chunk's A
constexpr int kOpABytes = kOpATile * 2;                       // 28 KiB
constexpr int kOpBBytes = kDigits * kOpCols * kTcK * 2;       // 3.5 KiB
constexpr int kOpSmemBytes = 2 * kOpABytes + 2 * kOpBBytes + 256;
constexpr int kOpSmemRequest = 70 * 1024;                     // three CTAs per SM

__global__ void op_identity_kernel(double2* __restrict__ G, int rows, int TS, int i0) {
  const size_t total = (size_t)rows * TS;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % TS), r = (int)(idx / TS);
    G[idx] = make_double2(c == i0 + r ? 1.0 : 0.0, 0.0);
  }
}

__global__ void op_collect_kernel(const double2* __restrict__ H, double* __restrict__ Op, int rows, int R, int TS, int i0) {
  const size_t total = (size_t)rows * R;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx % R), r = (int)(idx / R);
    if (i0 + r < TS) Op[(size_t)t * TS + i0 + r] = H[(size_t)r * TS + t].x;
  }
}

// One CTA per (row t, parity): Q_sigma[t][t'] for t' < R from Op; the diagonal entry into `diag`,
// the exponent bound of the off-diagonal entries and their digits (0 at t' = t) into the K-major
// tiles.
__global__ void __launch_bounds__(128) op_digits_kernel(const double* __restrict__ Op, unsigned short* __restrict__ dig,
                                                         int* __restrict__ rexp, double* __restrict__ diag, int R,
                                                         int TS, int L, int O, int nt, int nk) {
  const int t = blockIdx.x, par = blockIdx.y;       // par 0: sigma = +1, 1: sigma = -1
  const double sg = par ? -1.0 : 1.0;
  __shared__ int emax_s;
  if (threadIdx.x == 0) emax_s = -100000;
  __syncthreads();
  auto q_at = [&](int tp) {
    if (t >= R) return 0.0;
    const bool self = (tp == O - tp) || (TS == 2 * L && tp == 0);
    const double a = Op[(size_t)t * TS + tp];
    return self ? (par ? 0.0 : a) : fma(sg, Op[(size_t)t * TS + (O - tp)], a);
  };
  int e = -100000;
  for (int tp = threadIdx.x; tp < R; tp += blockDim.x) {
    const double q = q_at(tp);
    if (tp == t) diag[par * nt * kTcRings + t] = q;
    else if (q != 0.0) e = max(e, theta::exp_of(q));
  }
  if (t >= R && threadIdx.x == 0) diag[par * nt * kTcRings + t] = 0.0;
  e = __reduce_max_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0) atomicMax(&emax_s, e);
  __syncthreads();
  const int rho = (emax_s < -2000 ? 0 : emax_s) + 2;   // |Q[t][.]| < 2^(rho - 1)
  if (threadIdx.x == 0) rexp[par * nt * kTcRings + t] = rho;
  const int tt = t / kTcRings, row = t % kTcRings;
  for (int tp = threadIdx.x; tp < R; tp += blockDim.x) {
    const uint2 q = offset_digits(tp == t ? 0.0 : q_at(tp), rho);
    unsigned short* tile = dig + ((size_t)(par * nt + tt) * nk + tp / kTcK) * kOpATile;
#pragma unroll
    for (int i = 0; i < kDigits; ++i)
      tile[i * kTcRings * kTcK + kmajor_off(row, tp % kTcK) / 2] = digit_half(q, i);
  }
}

// cexp[s][r][part] = max over the rings of the exponent of F[s][t'][k(m)] (part 0 re, 1 im).
// Block = 32 consecutive rows of one signal x 8 groups of rings; a warp reads 32 consecutive
// spectrum entries of one ring.
__global__ void __launch_bounds__(256) op_colexp_kernel(const double2* __restrict__ F, int* __restrict__ cexp, int S,
                                                         int MR, int R, int FW, int mo) {
  __shared__ int red[8][32][2];
  const int rl = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int rblocks = (MR + 31) / 32;
  const int s = blockIdx.x / rblocks, r = (blockIdx.x % rblocks) * 32 + rl;
  int er = -100000, ei = -100000;
  if (r < MR) {
    const int m = r - mo, k = m >= 0 ? m : m + FW;
    const double2* col = F + (size_t)s * R * FW + k;
    for (int tp = grp; tp < R; tp += 8) {
      const double2 v = col[(size_t)tp * FW];
      if (v.x != 0.0) er = max(er, theta::exp_of(v.x));
      if (v.y != 0.0) ei = max(ei, theta::exp_of(v.y));
    }
  }
  red[grp][rl][0] = er;
  red[grp][rl][1] = ei;
  __syncthreads();
  if (grp == 0 && r < MR) {
    for (int q = 1; q < 8; ++q) {
      er = max(er, red[q][rl][0]);
      ei = max(ei, red[q][rl][1]);
    }
    cexp[2 * ((size_t)s * MR + r)] = er;
    cexp[2 * ((size_t)s * MR + r) + 1] = ei;
  }
}

__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

struct OpArgs {
  const double2* F;        // [S][R][FW] spectra
  double2* H;              // [S][MR][TS] output rows (t < R written)
  const int* cexp;         // [S][MR][2]
  const unsigned short* dig;
  const int* rexp;
  const double* diag;      // [2][nt * 128] Q_sigma[t][t]
  const int* n_of;
  int S, MR, R, FW, TS, mo, nN, L, nt, nk, mlo, mhi, ncol0;   // ncol0: column tiles per parity
};

// Grid: x = tile of 128 rings t, y = column tile (parity 0 first), z = signal.
__global__ void __launch_bounds__(kTcRings, 3) theta_operator_tc_kernel(OpArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tt = blockIdx.x, s = blockIdx.z;
  const int par = (int)blockIdx.y >= a.ncol0 ? 1 : 0;
  const int ct = (int)blockIdx.y - par * a.ncol0;
  const int n = a.n_of[s % a.nN];
  // orders of this parity class: m = mfirst, mfirst + 2, ...; this CTA's 8 of them
  const int mfirst = a.mlo + ((((a.mlo - n - par) % 2) + 2) % 2);
  const int m0 = mfirst + 2 * kOpCols / 2 * ct;
  if (m0 > a.mhi) return;

  unsigned char* sA = smem;                                   // [2][28 KiB]
  unsigned char* sB = smem + 2 * kOpABytes;                   // [2][3.5 KiB]
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + 2 * kOpBBytes);
  uint64_t* done = full + 2;
  int* ce_s = reinterpret_cast<int*>(done + 2);               // [16] column exponent bounds
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ce_s + kOpCols);
  int* abort_s = reinterpret_cast<int*>(tmem_slot + 1);

  const unsigned short* dig = a.dig + (size_t)(par * a.nt + tt) * a.nk * kOpATile;
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(tc::smem_addr(&full[q]), 1);
      tc::mbar_init(tc::smem_addr(&done[q]), 1);
    }
    tc::mbar_init_fence();
    *abort_s = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tmem_slot), kTmemCols);
  if (tid < kOpCols) {
    const int m = m0 + 2 * (tid >> 1);
    int e = -100000;
    if (m <= a.mhi) e = a.cexp[((size_t)s * a.MR + (m + a.mo)) * 2 + (tid & 1)];
    ce_s[tid] = (e < -2000 ? 0 : e) + 2;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sA_addr = tc::smem_addr(sA), sB_addr = tc::smem_addr(sB);
  if (tid == 0) bulk_copy_g2s(sA_addr, dig, kOpABytes, tc::smem_addr(&full[0]));

  // this thread's digit-split column and ring pair of every chunk (all 128 threads)
  const int bn = tid % kOpCols, bq = tid / kOpCols;
  const int bm = m0 + 2 * (bn >> 1);
  const bool bact = bm <= a.mhi;
  const int bk = bm >= 0 ? bm : bm + a.FW;
  const double2* Fs = a.F + (size_t)s * a.R * a.FW;

  long long X[kOpCols], Y[kOpCols];
#pragma unroll
  for (int c = 0; c < kOpCols; ++c) { X[c] = 0; Y[c] = 0; }
  int since_reset = 0;
  bool ok = true;
  for (int kc = 0; kc < a.nk; ++kc) {
    const int st = kc & 1;
    {
      uint2 q[2];
      const int ce = ce_s[bn];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int tp = kc * kTcK + 2 * bq + u;
        double v = 0.0;
        if (bact && tp < a.R) {
          const double* f = reinterpret_cast<const double*>(Fs + (size_t)tp * a.FW + bk);
          v = f[bn & 1];
        }
        q[u] = offset_digits(v, ce);
      }
      uint32_t w[kDigits];
      w[0] = digit_pair(q[0].y, q[1].y, 2);
      w[1] = digit_pair(q[0].y, q[1].y, 1);
      w[2] = digit_pair(q[0].y, q[1].y, 0);
      w[3] = digit_pair(q[0].x, q[1].x, 3);
      w[4] = digit_pair(q[0].x, q[1].x, 2);
      w[5] = digit_pair(q[0].x, q[1].x, 1);
      w[6] = digit_pair(q[0].x, q[1].x, 0);
      // this stage's previous MMAs (chunk kc - 2) must be done before it is rewritten
      if (kc >= 2 && !tc::mbar_wait(tc::smem_addr(&done[st]), (uint32_t)(((kc >> 1) - 1) & 1))) {
        set_status(tc::kStatusMmaWait);
        *abort_s = 1;
      }
      unsigned char* bst = sB + st * kOpBBytes;
#pragma unroll
      for (int i = 0; i < kDigits; ++i)
        *reinterpret_cast<uint32_t*>(bst + kmajor_off(kLevelCols * i + bn, 2 * bq)) = w[i];
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (*abort_s) { ok = false; break; }
    if (tid == 0) {
      if (!tc::mbar_wait(tc::smem_addr(&full[st]), (uint32_t)((kc >> 1) & 1))) {
        set_status(tc::kStatusMmaWait);
        *abort_s = 1;
      } else {
        tc::fence_after_sync();
#pragma unroll
        for (int i = 0; i < kDigits; ++i) {
          const uint64_t ad = tc::smem_desc(sA_addr + st * kOpABytes + i * kATileBytes, 128, 256);
          const uint64_t bd = tc::smem_desc(sB_addr + st * kOpBBytes, 128, 256);
          tc::mma_f16(tmem + kLevelCols * i, ad, bd, tc::idesc_f16_f32(kTcRings, kLevelCols * (kDigits - i)),
                      since_reset > 0 || i > 0);
        }
        tc::mma_commit(tc::smem_addr(&done[st]));
        // the next chunk's matrix digits into the other stage, once that stage's MMAs are done
        if (kc + 1 < a.nk) {
          const int sn = (kc + 1) & 1;
          if (kc >= 1 && !tc::mbar_wait(tc::smem_addr(&done[sn]), (uint32_t)((((kc + 1) >> 1) - 1) & 1))) {
            set_status(tc::kStatusMmaWait);
            *abort_s = 1;
          } else {
            bulk_copy_g2s(sA_addr + sn * kOpABytes, dig + (size_t)(kc + 1) * kOpATile, kOpABytes,
                          tc::smem_addr(&full[sn]));
          }
        }
      }
    }
    ++since_reset;
    if (since_reset == kDrainChunks || kc == a.nk - 1) {
      if (!tc::mbar_wait(tc::smem_addr(&done[st]), (uint32_t)((kc >> 1) & 1))) {
        set_status(tc::kStatusMmaWait);
        ok = false;
      }
      tc::fence_after_sync();
      if (__all_sync(0xffffffffu, ok)) {
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int lam[kDigits][8];
#pragma unroll
          for (int lv = 0; lv < kDigits; ++lv) {
            uint32_t r[8];
            tc::tmem_ld8(trow + (uint32_t)(kLevelCols * lv + 8 * h), r);
            tc::tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 8; ++e) lam[lv][e] = __float2int_rn(__uint_as_float(r[e]));
          }
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            X[8 * h + e] += ((long long)lam[0][e] << 24) + ((long long)lam[1][e] << 16) +
                            ((long long)lam[2][e] << 8) + (long long)lam[3][e];
            Y[8 * h + e] += ((long long)lam[4][e] << 16) + ((long long)lam[5][e] << 8) + (long long)lam[6][e];
          }
        }
      }
      tc::fence_before_sync();
      since_reset = 0;
      if (!__syncthreads_and(ok)) { ok = false; break; }
    }
  }
  // H[s][m + mo][t] = Q_sigma[t][t] F[s][t][k(m)] + 2^(rho_t + eps_c - 38) (X + 2^-24 Y), re and im
  const int t = tt * kTcRings + tid;
  if (ok && t < a.R) {
    const int rho = a.rexp[par * a.nt * kTcRings + t];
    const double qd = a.diag[par * a.nt * kTcRings + t];
#pragma unroll
    for (int o = 0; o < kOpCols / 2; ++o) {
      const int m = m0 + 2 * o;
      if (m > a.mhi) break;
      const double2 f = Fs[(size_t)t * a.FW + (m >= 0 ? m : m + a.FW)];
      const double re = ldexp(fma((double)Y[2 * o], 0x1p-24, (double)X[2 * o]), rho + ce_s[2 * o] - 38);
      const double im = ldexp(fma((double)Y[2 * o + 1], 0x1p-24, (double)X[2 * o + 1]), rho + ce_s[2 * o + 1] - 38);
      a.H[((size_t)s * a.MR + (m + a.mo)) * a.TS + t] = make_double2(fma(qd, f.x, re), fma(qd, f.y, im));
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

cudaError_t launch_theta_inverse_tc32(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (a.nsig >= 16) return launch_inv_tc32<16>(a, st);
  if (a.nsig >= 8) return launch_inv_tc32<8>(a, st);
  if (a.nsig >= 4) return launch_inv_tc32<4>(a, st);
  if (a.nsig >= 2) return launch_inv_tc32<2>(a, st);
  return launch_inv_tc32<1>(a, st);
}

cudaError_t launch_theta_inverse_tc(const Plan& p, const InvArgs& a, cudaStream_t st) {
  if (paired_plan(p)) {
    if (a.nsig >= 2) return launch_inv_tc<2, true>(a, st);
    return launch_inv_tc<1, true>(a, st);
  }
  if (a.nsig >= 4) return launch_inv_tc<4, false>(a, st);
  if (a.nsig >= 2) return launch_inv_tc<2, false>(a, st);
  return launch_inv_tc<1, false>(a, st);
}

// Forward theta stage on the tensor cores, for launches of at most 8 tiles of 256 rings (2048
// rings) written straight to flm; other launches return cudaErrorNotSupported.
cudaError_t launch_theta_forward_tc(const Plan& p, const FwdArgs& a, cudaStream_t st) {
  if (a.part || (a.nrows + kFwdRings - 1) / kFwdRings > kFwdMaxTiles) return cudaErrorNotSupported;
  if (paired_plan(p)) {
    if (a.nsig >= 2) return launch_fwd_tc<2, true>(a, st);
    return launch_fwd_tc<1, true>(a, st);
  }
  if (a.nsig >= 4) return launch_fwd_tc<4, false>(a, st);
  if (a.nsig >= 2) return launch_fwd_tc<2, false>(a, st);
  return launch_fwd_tc<1, false>(a, st);
}

cudaError_t launch_op_identity(void* G, int rows, int TS, int i0, cudaStream_t st) {
  op_identity_kernel<<<1024, 256, 0, st>>>(reinterpret_cast<double2*>(G), rows, TS, i0);
  return launched();
}

cudaError_t launch_op_collect(const void* H, double* Op, int rows, int R, int TS, int i0, cudaStream_t st) {
  op_collect_kernel<<<1024, 256, 0, st>>>(reinterpret_cast<const double2*>(H), Op, rows, R, TS, i0);
  return launched();
}

cudaError_t launch_op_digits(const Plan& p, const double* Op, cudaStream_t st) {
  const int O = p.sampling == S2GB_MWSS ? 2 * p.L : 2 * p.L - 2;
  op_digits_kernel<<<dim3(p.op_nt * kTcRings, 2), 128, 0, st>>>(Op, p.op_dig, p.op_rexp, p.op_diag, p.R, p.TS,
                                                               p.L, O, p.op_nt, p.op_nk);
  return launched();
}

cudaError_t launch_operator_tc(const Plan& p, const void* F, void* H, int* cexp, int S, cudaStream_t st) {
  static_assert(kOpSmemBytes <= kOpSmemRequest, "shared memory layout");
  OpArgs a;
  a.F = reinterpret_cast<const double2*>(F);
  a.H = reinterpret_cast<double2*>(H);
  a.cexp = cexp;
  a.dig = p.op_dig;
  a.rexp = p.op_rexp;
  a.diag = p.op_diag;
  a.n_of = p.n_of;
  a.S = S; a.MR = p.MR; a.R = p.R; a.TS = p.TS; a.nN = p.nN; a.L = p.L; a.nt = p.op_nt; a.nk = p.op_nk;
  a.FW = p.real ? p.L : p.P;
  a.mo = p.real ? 0 : p.L - 1;
  a.mlo = p.real ? 0 : -(p.L - 1);
  a.mhi = p.L - 1;
  a.ncol0 = (p.L + kOpCols / 2 - 1) / (kOpCols / 2);     // >= ceil(#orders of a parity / 8)
  op_colexp_kernel<<<S * ((p.MR + 31) / 32), 256, 0, st>>>(a.F, cexp, S, p.MR, p.R, a.FW, a.mo);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  e = set_dynamic_smem((const void*)theta_operator_tc_kernel, kOpSmemRequest);
  if (e != cudaSuccess) return e;
  theta_operator_tc_kernel<<<dim3(p.op_nt, 2 * a.ncol0, S), kTcRings, kOpSmemRequest, st>>>(a);
  return launched();
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
