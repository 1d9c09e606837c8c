// Internal declarations shared by the translation units of libs2gb.so.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/s2gb.h"

namespace s2gb {

// Rings whose sin(theta) is below this use the difference form of the l-recursion (see
// theta_kernels.cu): there the plain three-term recurrence amplifies rounding by ~1/sin(theta).
constexpr double kPoleSin = 0.15;

// Per-ring data, host-computed in extended precision and rounded once.
struct RingData {
  double v;        // 2 sin^2(theta/2) for north rings (theta < pi/2), 2 cos^2(theta/2) for south
  double ls_hi;    // log2 sin(theta/2) as an unevaluated double-double (hi + lo)
  double ls_lo;
  double lc_hi;    // log2 cos(theta/2) (lc_hi = -inf at theta = pi)
  double lc_lo;
  int north;       // theta < pi/2
  int pole;        // 1: theta == pi (cos(theta/2) = 0), 2: theta == 0 (sin(theta/2) = 0), else 0
  int diff;        // sin(theta) < kPoleSin: difference form of the recursion
  int pad;
};

// Per (n, m) data of the starting value d^{l0}_{m,n}, l0 = max(|m|,|n|) (Eq. "initial_values"
// plus the symmetries of Sec. 3.3): d = sign * 2^{p} * sin(theta/2)^a * cos(theta/2)^b with
// p = log2 sqrt((2 l0)! / (a! b!)), a + b = 2 l0.
struct SeedData {
  double p_hi;
  double p_lo;
  int l0;
  int a;
  int b;
  int sign;
};

// Recursion step j -> j+1 coefficients for one (n, m), see theta_kernels.cu.
constexpr int kCoefPerStep = 6;  // A, C, K_north, K_south, Kd_north, Kd_south (float32 kernels)
// Normalised form used by the float64 kernels (plan.cu, coefn_kernel):
// A', K_n', K_s', gamma_j, gamma_{j+1}, A'', Kd_n'', Kd_s'', eta_{j+1}, 1/gamma_j
constexpr int kCoefPerStepN = 10;
constexpr int kFwdChunk = 2048;  // rings per CTA of the forward theta kernel
constexpr int kOpMaxRings = 2304;  // rings up to which the theta-direction operator is a matrix

struct Plan {
  int L = 0, spin = 0, N = 0, precision = 0, max_batch = 0, device = 0;
  int sampling = S2GB_MW;
  int T = 0;        // 2L - 1 (number of orders)
  int R = 0;        // theta rings of the sampling: L (MW), L + 1 (MWSS), 2L (DH)
  int P = 0;        // phi samples per ring: 2L - 1 (MW, DH), 2L (MWSS)
  int TS = 0;       // theta-torus length of the forward quadrature operator: 2L - 1 (MW), 2L
                    // (MWSS), 0 (DH: explicit ring weights, no operator)
  int nN = 1;       // number of n values (1 for the sphere, 2N-1 for Wigner)
  int Nfft = 0;     // length of the fine theta grid of the forward quadrature (>= 4L-3)
  int ring0 = 0;    // the recursion kernels run over the rings [ring0, ring0 + nint): all of them
  int nint = 0;     // on MW and DH; on MWSS the interior (the two pole rings, where d is a
                    // Kronecker delta, are handled by the pole kernels), likewise MW's ring theta = pi
                    // with the order recursion (its lambda_m has 1/sin(theta))
  int pole_n = -1;  // ring index of theta = 0 handled by the pole kernels, or -1
  int pole_s = -1;  // ring index of theta = pi handled by the pole kernels, or -1
  bool mrec = false;  // theta stages by the recursion over the order m (theta_mrec.cu)
  bool tc = false;    // float64 on-the-fly plans: the theta contraction on the tensor cores
  bool tc32 = false;  // float32 plans of max_batch >= 16: the inverse contraction on the tensor cores
                      // (theta_tc.cu); false: on the float64 FMA pipe (theta_kernels.cu)
  // The forward's theta-direction quadrature operator (torus extension, then the FFT operator of
  // api.cu's theta_weight_operator, restricted to the R rings) is linear and the same for every
  // order row up to the parity sigma = (-1)^(m-n): two real R x R matrices Q_sigma.  Tensor-core MW /
  // MWSS plans with R <= kOpMaxRings keep them as float16 digit tiles and apply them on the tensor
  // cores (theta_tc.cu) instead of the FFTs.
  bool tc_op = false;
  unsigned short* op_dig = nullptr;   // [2][op_nt][op_nk][7][128 x 16] K-major digit tiles
  int* op_rexp = nullptr;             // [2][op_nt * 128]: |E_sigma[t][.]| < 2^(op_rexp - 1)
  double* op_diag = nullptr;          // [2][op_nt * 128]: Q_sigma[t][t] (0 past R)
  int op_nt = 0, op_nk = 0;           // 128-row tiles over t, 16-column chunks over t'
  int cap_n = 0;    // rings [ring0, cap_n) and [cap_s, ring0 + nint) use the difference form
  int cap_s = 0;
  int fwd_parts = 1;  // forward theta stage in one launch (nint <= kFwdChunk) or in ring chunks
  bool wigner = false;
  bool real = false;  // real signals (spin 0): orders m >= 0 only, f real, flm [L][L]
  int MR = 0;         // order rows of the theta-direction buffers: T (complex) or L (real)

  // device tables
  double* coef = nullptr;      // [nN][T][L][kCoefPerStepN] (m index = m + L - 1, step j); FP64 plans
  float* coef32 = nullptr;     // the same table rounded to float (FP32 plans)
  float* v32 = nullptr;        // [R] ring variable v rounded to float (FP32 plans)
  RingData* ring = nullptr;    // [R]
  SeedData* seed = nullptr;    // [nN][T]
  double* scale_inv = nullptr; // [nN][L] per-degree factor of the inverse theta stage
  double* scale_fwd = nullptr; // [nN][L] per-degree factor of the forward theta stage
  double* wfine = nullptr;     // [Nfft] weights on the fine grid (constants folded in)
  double* nu = nullptr;        // [R] ring weights of the forward quadrature: fold factors
                               // (MW 2, ..., 2, 1; MWSS 1, 2, ..., 2, 1) or DH weights * 2 pi/P
  int* n_of = nullptr;         // [nN] n for each n index
  double* mrec_ab = nullptr;   // [L][T] (a_{m-1}, a_{m-1}/a_m) of the order recursion (mrec plans)
  double* csc = nullptr;       // [R] 1/sin(theta) of the interior rings (mrec plans)
  size_t device_bytes = 0;

  // precompute mode (FP64, L <= kFwdChunk): d^l_{m,n}(theta_t) of every (n, m) theta kernels run,
  // rows l = l0 .. L-1 of L doubles (t fastest), zero where the on-the-fly kernels would skip a
  // chain as dead (|d| < 2^-kLiveThr)
  bool precompute = false;
  double* dtab = nullptr;
  size_t* tab_off = nullptr;   // [nN][T] offset (doubles) of the rows of (n, m), kNoTable if none
  int* live0 = nullptr;        // [nN][T][ceil(L/32)] first degree with a live chain in 32 rings

  // cuFFT plans: index 0 = one signal, 1 = max_batch signals (rows of the whole batch)
  cufftHandle fft_phi[2] = {0, 0};   // length P along rows of length P, S*R rows (real: R2C)
  cufftHandle fft_phi_c2r[2] = {0, 0};   // real plans: the inverse direction (C2R)
  cufftHandle fft_T[2] = {0, 0};     // length TS, S*MR rows (MW, MWSS)
  cufftHandle fft_N[2] = {0, 0};     // length Nfft, S*MR rows (MW, MWSS)
  cufftHandle fft_gam[1] = {0};      // length 2N-1, stride R*P, R*P rows (one signal)
  bool fft_made[2] = {false, false};
  bool fft_op_made[2] = {false, false};   // fft_T / fft_N exist (TS > 0)
  bool fft_gam_made = false;
  size_t fft_work = 0;               // max cuFFT work area over all plans
  std::mutex fft_mutex;
};

// ---- kernels (theta_kernels.cu) ----
struct InvArgs {
  const void* flm;      // [S][L][T] coefficients (S = batch * nN signals)
  void* out;            // output with strides below
  long long s_sig;      // stride between signals in out (elements)
  long long s_t;        // stride between rings
  long long s_m;        // stride between orders
  int m_mod;            // 1: column = m mod mmod, 0: column = m + L - 1
  int mmod;             // P (the phi DFT length)
  int nsig;             // number of signals per n (batch)
  int nN;
  int L;
  int ring0;            // the recursion kernel's rings: [ring0, nring)
  int nring;
  const double* coef;
  const RingData* ring;
  const SeedData* seed;
  const double* scale;  // [nN][L]
  const float* coef32;  // FP32 plans
  const float* v32;
  const double* dtab;   // precompute mode (else null): the d table, its offsets, live starts
  const size_t* tab_off;
  const int* live0;
  int rank0;            // orders of this launch: m-ranks [rank0, rank0 + nrank) (m_of_rank order
  int nrank;            // 0, -1, 1, -2, 2, ...: |m| in [lo, hi) is ranks [max(0, 2lo-1), 2hi-1))
  int mpos;             // 1: rank r is order m = r (real-signal plans: m >= 0 only)
  int flm_ld;           // row length of flm (T; L for real-signal plans)
  int flm_c0;           // column of m = 0 in flm (L - 1; 0 for real-signal plans)
  void* mpart;          // order-recursion plans: workspace for the per-CTA partial sums
};

struct FwdArgs {
  const void* g;        // input with strides below
  void* flm;            // [S][L][T]
  long long s_sig, s_t, s_m;
  int m_mod;            // as in InvArgs
  int mmod;
  int use_nu;           // multiply g by the ring weights nu_t
  int nsig;
  int nN;
  int L;
  const double* coef;
  const RingData* ring;
  const SeedData* seed;
  const double* scale;
  const double* nu;
  const float* coef32;  // FP32 plans
  const float* v32;
  const double* dtab;   // precompute mode (as in InvArgs)
  const size_t* tab_off;
  const int* live0;
  int row0;             // ring range of this launch: [row0, row0 + nrows)
  int nrows;
  void* part;           // non-null: write this launch's partial result at part + part_off
  long long part_off;   // (elements) instead of flm; a fixed-order sum of the parts gives flm
  int rank0;            // orders of this launch (as in InvArgs)
  int nrank;
  int mpos;             // flm layout and order mapping as in InvArgs
  int flm_ld;
  int flm_c0;
  void* mpart;          // order-recursion plans: workspace for the per-CTA partial sums
};

// Arguments of the order-recursion kernels (theta_mrec.cu)
struct MrecArgs {
  const double2* ab;    // [L][T] (a_{m-1}, a_{m-1}/a_m)
  const double* csc;    // [R] 1/sin(theta)
  const int* n_of;
  void* part;           // partial sums
  int nint;             // rings of the recursion
  int mlo, mhi;         // orders |m| in [mlo, mhi) are written
  int mlow1;            // forward: lowest order of the CTA's first sweep
};
cudaError_t launch_theta_inverse_mrec(const Plan& p, const InvArgs& a, cudaStream_t st);
cudaError_t launch_theta_forward_mrec(const Plan& p, const FwdArgs& a, cudaStream_t st);
size_t mrec_part_bytes(const Plan& p, int batch);   // workspace region D of order-recursion plans

// m-ranks of the orders with |m| in [lo, hi), 0 <= lo <= hi <= L (empty: count 0)
inline void mrange_ranks(int lo, int hi, int& rank0, int& nrank) {
  rank0 = lo == 0 ? 0 : 2 * lo - 1;
  const int end = hi == 0 ? 0 : 2 * hi - 1;
  nrank = end > rank0 ? end - rank0 : 0;
}

// Every launcher returns launched(): it counts one launch of this library's kernels (a host-side,
// process-wide counter read by s2gb_kernels_launched) and returns cudaGetLastError().
cudaError_t launched();
// sets a kernel's dynamic shared-memory limit, once per (kernel, device) and size (api.cu)
cudaError_t set_dynamic_smem(const void* func, size_t bytes);

cudaError_t launch_theta_inverse(const Plan& p, const InvArgs& a, cudaStream_t st);
// MWSS pole rings theta = 0 and pi (Sec. 3.3: d^l_{mn}(0) = delta_{mn}, d^l_{mn}(pi) =
// (-1)^{l-n} delta_{m,-n}): the inverse-shaped stage writes both rings for the launch's orders,
// the forward-shaped stage adds their terms to flm (after the interior rings' kernel)
cudaError_t launch_pole_inverse(const Plan& p, const InvArgs& a, cudaStream_t st);
cudaError_t launch_pole_forward(const Plan& p, const FwdArgs& a, cudaStream_t st);
// precompute mode (theta_precompute.cu): table construction at plan creation, and the theta stages
// reading it
constexpr size_t kNoTable = ~(size_t)0;
// Pairing (m, n) with (-m, -n) needs the set of n to be symmetric: spin-0 sphere plans and Wigner
// (real-signal plans have the orders m >= 0 only and need no partner).
inline bool paired_plan(const Plan& p) { return !p.real && (p.wigner || p.spin == 0); }
int build_dtable(Plan* p, size_t* bytes);
cudaError_t launch_theta_inverse_pre(const Plan& p, const InvArgs& a, cudaStream_t st);
cudaError_t launch_theta_forward_pre(const Plan& p, const FwdArgs& a, cudaStream_t st);
cudaError_t launch_theta_forward(const Plan& p, const FwdArgs& a, cudaStream_t st);
cudaError_t launch_theta_inverse_f32(const Plan& p, const InvArgs& a, cudaStream_t st);
// float64 theta stages with the contraction on the tensor cores (theta_tc.cu)
cudaError_t launch_theta_inverse_tc(const Plan& p, const InvArgs& a, cudaStream_t st);
cudaError_t launch_theta_inverse_tc32(const Plan& p, const InvArgs& a, cudaStream_t st);
cudaError_t launch_theta_forward_tc(const Plan& p, const FwdArgs& a, cudaStream_t st);
// plan creation: the operator matrices from the operator's responses (theta_tc.cu)
//   op_identity: rows r < rows of G [rows][TS] = unit vectors at torus points i0 + r
//   op_collect:  Op[t][i0 + r] = Re H[r][t] for t < R
//   op_digits:   Q_sigma rows from Op (R x TS); the diagonal into op_diag, the off-diagonal part
//                E_sigma as exponents and digit tiles into the plan
cudaError_t launch_op_identity(void* G, int rows, int TS, int i0, cudaStream_t st);
cudaError_t launch_op_collect(const void* H, double* Op, int rows, int R, int TS, int i0, cudaStream_t st);
cudaError_t launch_op_digits(const Plan& p, const double* Op, cudaStream_t st);
// forward: H[s][m + mo][t] (t < R, rows of TS) = sum_t' Q_sigma[t][t'] F[s][t'][k(m)], with the
// per-column exponents in `cexp` ([S][MR][2] ints of scratch)
cudaError_t launch_operator_tc(const Plan& p, const void* F, void* H, int* cexp, int S, cudaStream_t st);
cudaError_t launch_theta_forward_f32(const Plan& p, const FwdArgs& a, cudaStream_t st);

// ---- glue kernels (glue.cu) ----
cudaError_t launch_extend(const Plan& p, const void* F, void* G, int nsig, cudaStream_t st);
cudaError_t launch_extend_adjoint(const Plan& p, const void* G, void* F, int nsig, cudaStream_t st);
cudaError_t launch_pad(const Plan& p, const void* X, void* Y, int rows, cudaStream_t st);
cudaError_t launch_truncate(const Plan& p, const void* Y, void* X, int rows, cudaStream_t st);
cudaError_t launch_weight_fine(const Plan& p, void* Y, int rows, cudaStream_t st);
cudaError_t launch_nu_extend(const Plan& p, void* X, int rows, cudaStream_t st);
// ring spectra [nsig][R][W]: ring t times nu_t (adjoint of the DH forward's ring weights)
cudaError_t launch_ring_weight(const Plan& p, void* X, int nsig, int W, cudaStream_t st);
// ring spectra [nsig][R][P] of MWSS plans: column L (the phi frequency no order owns) set to 0
cudaError_t zero_nyquist(const Plan& p, void* X, int nsig, cudaStream_t st);
// out[i] = sum of the parts in order, for the columns (c0 + m, rows of ld) of orders |m| in [mlo, mhi)
cudaError_t launch_sum_parts(const Plan& p, const void* parts, void* out, int nsig, int nparts,
                             int mlo, int mhi, int ld, int c0, cudaStream_t st);
// real-signal spectra [rows][L]: columns m >= 1 times s, imaginary part of column 0 dropped
cudaError_t launch_scale_nonzero_orders(const Plan& p, void* X, size_t rows, double s, cudaStream_t st);
cudaError_t launch_gamma_reorder(const Plan& p, const void* in, void* out, int batch, int to_signal,
                                 double scale, cudaStream_t st);

// ---- plan helpers (plan.cu) ----
int make_plan(Plan* p);
void free_plan(Plan* p);
size_t workspace_bytes(const Plan& p, int batch);
void workspace_regions(const Plan& p, int batch, size_t out[4]);   // bytes of regions A, B, C, D

}  // namespace s2gb
