// C ABI of libs2gb.so (declared in include/s2gb.h): argument checks and the stage sequences of
// the transforms.  Every stage runs on the caller's stream; nothing here allocates after plan
// creation.
//
// Forward, per signal (Sec. 4.1 and 4.2.2), with T = 2L-1 and NF >= 4L-3:
//   F   = DFT_T along phi                                  (Eq. disc_sh_fft, without q_Phi)
//   G   = torus extension of F in theta (order-major rows of length T)
//   H   = (1/(T NF)) IDFT_T . trunc . DFT_N . W . IDFT_N . pad . DFT_T (G)
//   flm = c_l sum_{t<L} d^l_{m,-s}(theta_t) nu_t H_m(theta_t)   (theta kernel, Eq. disc_sh_expanded)
// H is the degree-(L-1) projection of G(theta) |sin theta|/2 on the theta torus, evaluated on the L
// MW rings: W holds that weight's Fourier series (|k| <= 2L-2) sampled on the fine grid
// x_j = pi/T + 2 pi j/NF (the half-sample shift cancels the phases of the MW grid), together with
// the constants (2 pi/T)^2/(T NF).  Because the d-functions are trigonometric polynomials of degree
// <= L-1 in theta, int_0^pi G d sin = int_torus H d |sin|/2... = (2pi/T) sum over the torus of H d,
// folded onto the L rings with nu_t = 2 (t < L-1) and nu_{L-1} = 1.  This integrates exactly what
// the upsample-to-2L route of Sec. 4.2.2 integrates, on L rings instead of 2L.
// MWSS (Sec. 4.2.2, L+1 rings with both poles, P = 2L phi samples): the same construction on a
// torus of TS = 2L points starting at theta = 0 (fine grid unshifted, the Nyquist frequency L of
// the 2L-point DFTs dropped), fold factors 1 on the two poles and 2 elsewhere.  DH (Sec. 4.2.1,
// 2L rings): no torus operator -- the theta kernel applies the DH weights times 2 pi/P to the phi
// spectra directly.
// Inverse (Eqs. disc_ish_expanded, disc_ish_fft): theta kernel into [t][m mod P], then IDFT_P
// (P = T on MW and DH).
// Wigner (Sec. 2.3, 4.5): a gamma DFT (forward, scaled by 2 pi/(2N-1)) or IDFT (inverse) around
// 2N-1 spin-(-n) stages, with per-degree factors 1 (forward) and (2l+1)/(8 pi^2) (inverse).
// Adjoints (Sec. 5.2): every stage transposed in reverse order; the operator between the two
// DFT_T calls above is self-adjoint, the theta kernels swap roles.
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "s2gb_internal.h"

struct s2gb_plan_s {
  s2gb::Plan p;
};

namespace s2gb {

static std::atomic<unsigned long long> g_kernel_launches{0};

cudaError_t launched() {
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (kernel, device) and size: later calls
// that need no larger size do not touch the runtime, so transforms can be captured into CUDA graphs
// once they have run (the attribute is not a stream operation).
cudaError_t set_dynamic_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, size_t>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.first.first == func && d.first.second == dev) {
      if (bytes <= d.second) return cudaSuccess;
      e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e == cudaSuccess) d.second = bytes;
      return e;
    }
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.push_back({{func, dev}, bytes});
  return e;
}

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Workspace {
  char* A;
  char* B;
  char* C;
  void* fft;
  char* D = nullptr;   // partial results of the chunked forward theta stage (L > kFwdChunk)
};

Workspace carve(const Plan& p, void* ws, int batch) {
  size_t r[4];
  workspace_regions(p, batch, r);
  const size_t a = align256(r[0]), b = align256(r[1]), c = align256(r[2]), d = align256(r[3]);
  char* base = reinterpret_cast<char*>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  Workspace w = {base, base + a, base + a + b, base + a + b + c + d};
  w.D = d ? base + a + b + c : nullptr;
  return w;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? S2GB_OK : S2GB_ECUDA; }

// Run one cuFFT plan over the whole batch (q = 1) or item by item (q = 0).
struct FftRunner {
  Plan& p;
  cudaStream_t st;
  void* work;
  int batch;
  int run(cufftHandle* hs, const void* in, void* out, size_t item_elems, int dir) {
    const bool whole = (batch == p.max_batch);
    const int q = whole ? 1 : 0;
    cufftHandle h = hs[q];
    if (cufftSetStream(h, st) != CUFFT_SUCCESS) return S2GB_ECUFFT;
    if (cufftSetWorkArea(h, work) != CUFFT_SUCCESS) return S2GB_ECUFFT;
    const int reps = whole ? 1 : batch;
    const size_t es = p.precision == S2GB_FP64 ? 16 : 8;
    for (int r = 0; r < reps; ++r) {
      const char* i = reinterpret_cast<const char*>(in) + r * item_elems * es;
      char* o = reinterpret_cast<char*>(out) + r * item_elems * es;
      cufftResult res;
      if (p.precision == S2GB_FP64)
        res = cufftExecZ2Z(h, (cufftDoubleComplex*)i, (cufftDoubleComplex*)o, dir);
      else
        res = cufftExecC2C(h, (cufftComplex*)i, (cufftComplex*)o, dir);
      if (res != CUFFT_SUCCESS) return S2GB_ECUFFT;
    }
    return S2GB_OK;
  }
  // Real-signal plans: rings of T real samples -> orders 0..L-1 (dir > 0) or back (dir < 0);
  // in_elems / out_elems are one signal's element counts (real or complex as the direction says).
  int run_real(cufftHandle* hs, const void* in, void* out, size_t in_elems, size_t out_elems, int dir) {
    const bool whole = (batch == p.max_batch);
    cufftHandle h = hs[whole ? 1 : 0];
    if (cufftSetStream(h, st) != CUFFT_SUCCESS) return S2GB_ECUFFT;
    if (cufftSetWorkArea(h, work) != CUFFT_SUCCESS) return S2GB_ECUFFT;
    const int reps = whole ? 1 : batch;
    const size_t rs = p.precision == S2GB_FP64 ? 8 : 4;       // bytes of one real
    const size_t ies = dir > 0 ? rs : 2 * rs, oes = dir > 0 ? 2 * rs : rs;
    for (int r = 0; r < reps; ++r) {
      const char* i = reinterpret_cast<const char*>(in) + r * in_elems * ies;
      char* o = reinterpret_cast<char*>(out) + r * out_elems * oes;
      cufftResult res;
      if (p.precision == S2GB_FP64)
        res = dir > 0 ? cufftExecD2Z(h, (cufftDoubleReal*)i, (cufftDoubleComplex*)o)
                      : cufftExecZ2D(h, (cufftDoubleComplex*)i, (cufftDoubleReal*)o);
      else
        res = dir > 0 ? cufftExecR2C(h, (cufftReal*)i, (cufftComplex*)o)
                      : cufftExecC2R(h, (cufftComplex*)i, (cufftReal*)o);
      if (res != CUFFT_SUCCESS) return S2GB_ECUFFT;
    }
    return S2GB_OK;
  }
};

#define S2GB_TRY(expr)            \
  do {                            \
    int _rc = (expr);             \
    if (_rc != S2GB_OK) return _rc; \
  } while (0)

InvArgs inv_args(const Plan& p, const void* flm, void* out, int batch, const double* scale,
                 long long s_sig, long long s_t, long long s_m, int m_mod) {
  InvArgs a;
  a.flm = flm; a.out = out; a.s_sig = s_sig; a.s_t = s_t; a.s_m = s_m; a.m_mod = m_mod;
  a.mmod = p.P;
  a.nsig = batch; a.nN = p.nN; a.L = p.L; a.ring0 = p.ring0; a.nring = p.ring0 + p.nint;
  a.coef = p.coef; a.ring = p.ring; a.seed = p.seed;
  a.scale = scale; a.coef32 = p.coef32; a.v32 = p.v32;
  a.dtab = p.dtab; a.tab_off = p.tab_off; a.live0 = p.live0;
  a.rank0 = 0; a.nrank = p.MR;
  a.mpos = p.real ? 1 : 0; a.flm_ld = p.MR; a.flm_c0 = p.real ? 0 : p.L - 1;
  a.mpart = nullptr;
  return a;
}

// CTAs of the orders |m| in [lo, hi): m-ranks of the 0, -1, 1, ... order, or m itself for
// real-signal plans (m >= 0 only).
void order_ranks(const Plan& p, int lo, int hi, int& rank0, int& nrank) {
  if (p.real) {
    rank0 = lo;
    nrank = hi > lo ? hi - lo : 0;
  } else {
    mrange_ranks(lo, hi, rank0, nrank);
  }
}

FwdArgs fwd_args(const Plan& p, const void* g, void* flm, int batch, const double* scale,
                 long long s_sig, long long s_t, long long s_m, int m_mod, int use_nu) {
  FwdArgs a;
  a.g = g; a.flm = flm; a.s_sig = s_sig; a.s_t = s_t; a.s_m = s_m; a.m_mod = m_mod; a.use_nu = use_nu;
  a.mmod = p.P;
  a.nsig = batch; a.nN = p.nN; a.L = p.L; a.coef = p.coef; a.ring = p.ring; a.seed = p.seed;
  a.scale = scale; a.nu = p.nu; a.coef32 = p.coef32; a.v32 = p.v32;
  a.row0 = p.ring0; a.nrows = p.nint; a.part = nullptr; a.part_off = 0;
  a.dtab = p.dtab; a.tab_off = p.tab_off; a.live0 = p.live0;
  a.rank0 = 0; a.nrank = p.MR;
  a.mpos = p.real ? 1 : 0; a.flm_ld = p.MR; a.flm_c0 = p.real ? 0 : p.L - 1;
  a.mpart = nullptr;
  return a;
}

// G (theta-torus rows of length TS, S*MR rows, in B) -> H in B, using A as the fine-grid buffer
// (MW and MWSS plans).
int theta_weight_operator(Plan& p, FftRunner& fr, char* A, char* B, int S) {
  const size_t rows_item = (size_t)p.nN * p.MR;
  const int rows = S * p.MR;
  cudaStream_t st = fr.st;
  S2GB_TRY(fr.run(p.fft_T, B, B, rows_item * p.TS, CUFFT_FORWARD));
  S2GB_TRY(cuda_rc(launch_pad(p, B, A, rows, st)));
  S2GB_TRY(fr.run(p.fft_N, A, A, rows_item * p.Nfft, CUFFT_INVERSE));
  S2GB_TRY(cuda_rc(launch_weight_fine(p, A, rows, st)));
  S2GB_TRY(fr.run(p.fft_N, A, A, rows_item * p.Nfft, CUFFT_FORWARD));
  S2GB_TRY(cuda_rc(launch_truncate(p, A, B, rows, st)));
  S2GB_TRY(fr.run(p.fft_T, B, B, rows_item * p.TS, CUFFT_INVERSE));
  return S2GB_OK;
}

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Gamma DFT of the Wigner transform, one signal at a time: [b][k][plane] -> [b][k'][plane] (dir
// CUFFT_FORWARD) or back (CUFFT_INVERSE); plane = R * P.
int gamma_dft(Plan& p, const void* in, void* out, int batch, void* work, cudaStream_t st, int dir) {
  if (cufftSetStream(p.fft_gam[0], st) != CUFFT_SUCCESS) return S2GB_ECUFFT;
  if (cufftSetWorkArea(p.fft_gam[0], work) != CUFFT_SUCCESS) return S2GB_ECUFFT;
  const size_t es = p.precision == S2GB_FP64 ? 16 : 8;
  const size_t plane = (size_t)p.R * p.P;
  for (int b = 0; b < batch; ++b) {
    const char* i = reinterpret_cast<const char*>(in) + (size_t)b * p.nN * plane * es;
    char* o = reinterpret_cast<char*>(out) + (size_t)b * p.nN * plane * es;
    cufftResult r = p.precision == S2GB_FP64
        ? cufftExecZ2Z(p.fft_gam[0], (cufftDoubleComplex*)i, (cufftDoubleComplex*)o, dir)
        : cufftExecC2C(p.fft_gam[0], (cufftComplex*)i, (cufftComplex*)o, dir);
    if (r != CUFFT_SUCCESS) return S2GB_ECUFFT;
  }
  return S2GB_OK;
}

// The forward's theta-direction operator as matrices (tensor-core MW / MWSS plans, R <=
// kOpMaxRings): the responses of the FFT operator above to unit vectors at every torus point give
// Op (R x TS, the rows t < R the theta kernel reads); the torus extension then folds Op into the
// two R x R matrices Q_sigma.  Q_sigma is close to diagonal (about |sin theta_t| times the
// quadrature step on the diagonal, off-diagonal rows some 1e-3 of it away from the poles), and the
// digit GEMM's error per term is set by the row's largest entry, so the diagonal is kept in
// float64 (op_diag, applied in the GEMM's epilogue) and only the off-diagonal part E_sigma goes to
// float16 digit tiles with one exponent per row.
int build_theta_operator(Plan& p) {
  if (!p.tc || p.TS == 0 || p.R > kOpMaxRings) return S2GB_OK;
  p.op_nt = (p.R + 127) / 128;
  p.op_nk = (p.R + 15) / 16;
  const size_t dig_bytes = (size_t)2 * p.op_nt * p.op_nk * 7 * 128 * 16 * sizeof(unsigned short);
  const size_t rexp_bytes = (size_t)2 * p.op_nt * 128 * sizeof(int);
  const size_t diag_bytes = (size_t)2 * p.op_nt * 128 * sizeof(double);
  if (cudaMalloc((void**)&p.op_dig, dig_bytes) != cudaSuccess) return S2GB_ENOMEM;
  if (cudaMalloc((void**)&p.op_rexp, rexp_bytes) != cudaSuccess) return S2GB_ENOMEM;
  if (cudaMalloc((void**)&p.op_diag, diag_bytes) != cudaSuccess) return S2GB_ENOMEM;
  if (cudaMemset(p.op_dig, 0, dig_bytes) != cudaSuccess) return S2GB_ECUDA;
  void* tmp = nullptr;
  double* Op = nullptr;
  const size_t wsb = workspace_bytes(p, 1);
  if (cudaMalloc(&tmp, wsb) != cudaSuccess) return S2GB_ENOMEM;
  if (cudaMalloc((void**)&Op, (size_t)p.R * p.TS * sizeof(double)) != cudaSuccess) {
    cudaFree(tmp);
    return S2GB_ENOMEM;
  }
  int rc = S2GB_OK;
  {
    const Workspace w = carve(p, tmp, 1);
    FftRunner fr{p, 0, w.fft, 1};
    const int rows = p.nN * p.MR;
    for (int i0 = 0; i0 < p.TS && rc == S2GB_OK; i0 += rows) {
      rc = cuda_rc(launch_op_identity(w.B, rows, p.TS, i0, 0));
      if (rc == S2GB_OK) rc = theta_weight_operator(p, fr, w.A, w.B, p.nN);
      if (rc == S2GB_OK) rc = cuda_rc(launch_op_collect(w.B, Op, rows, p.R, p.TS, i0, 0));
    }
    if (rc == S2GB_OK) rc = cuda_rc(launch_op_digits(p, Op, 0));
    if (rc == S2GB_OK && cudaDeviceSynchronize() != cudaSuccess) rc = S2GB_ECUDA;
  }
  cudaFree(Op);
  cudaFree(tmp);
  if (rc != S2GB_OK) return rc;
  p.tc_op = true;
  p.device_bytes += dig_bytes + rexp_bytes + diag_bytes;
  return S2GB_OK;
}

// Scratch for the operator's per-column exponents: past the spectra in region A.
int* operator_cexp(const Plan& p, const Workspace& w, int S, size_t fw) {
  return reinterpret_cast<int*>(w.A + align256((size_t)S * p.R * fw * 16));
}

// Orders |m| in [mlo, mhi) of the forward transform: every stage before the theta kernel runs in
// full, the theta kernel only for those orders (flm entries of other orders are not written).
// MW / MWSS: phi DFT, torus extension, theta-direction quadrature operator, theta kernel over the
// rings with the fold factors.  DH: phi DFT, theta kernel over the rings with the DH weights.
int do_forward(Plan& p, const void* f, void* flm, int batch, const Workspace& w, cudaStream_t st,
               int mlo, int mhi) {
  FftRunner fr{p, st, w.fft, batch};
  const int S = batch * p.nN;
  const size_t plane = (size_t)p.R * p.P;
  const void* sig_in = f;
  if (p.wigner) {
    S2GB_TRY(gamma_dft(p, f, w.C, batch, w.fft, st, CUFFT_FORWARD));
    S2GB_TRY(cuda_rc(launch_gamma_reorder(p, w.C, w.B, batch, 1, kTwoPi / (2 * p.N - 1), st)));
    sig_in = w.B;
  }
  S2GB_TRY(fr.run(p.fft_phi, sig_in, w.A, (size_t)p.nN * plane, CUFFT_FORWARD));
  FwdArgs a;
  if (p.sampling == S2GB_DH) {
    a = fwd_args(p, w.A, flm, batch, p.scale_fwd, (long long)plane, p.P, 1, 1, 1);
  } else {
    if (p.tc_op) {
      S2GB_TRY(cuda_rc(launch_operator_tc(p, w.A, w.B, operator_cexp(p, w, S, p.P), S, st)));
    } else {
      S2GB_TRY(cuda_rc(launch_extend(p, w.A, w.B, S, st)));
      S2GB_TRY(theta_weight_operator(p, fr, w.A, w.B, S));
    }
    a = fwd_args(p, w.B, flm, batch, p.scale_fwd, (long long)p.MR * p.TS, 1, p.TS, 0, 1);
  }
  a.part = w.D;
  a.mpart = w.D;
  order_ranks(p, mlo, mhi, a.rank0, a.nrank);
  return cuda_rc(launch_theta_forward(p, a, st));
}

// Sphere inverse after the theta stage: ring spectra [b][t][m mod P] -> f (Eq. disc_ish_fft).
int do_inverse_phi(Plan& p, const void* ftilde, void* f, int batch, const Workspace& w, cudaStream_t st) {
  FftRunner fr{p, st, w.fft, batch};
  return fr.run(p.fft_phi, ftilde, f, (size_t)p.R * p.P, CUFFT_INVERSE);
}

int do_inverse(Plan& p, const void* flm, void* f, int batch, const Workspace& w, cudaStream_t st) {
  FftRunner fr{p, st, w.fft, batch};
  const size_t plane = (size_t)p.R * p.P;
  InvArgs a = inv_args(p, flm, w.A, batch, p.scale_inv, (long long)plane, p.P, 1, 1);
  a.mpart = w.D;
  S2GB_TRY(cuda_rc(launch_theta_inverse(p, a, st)));
  S2GB_TRY(cuda_rc(zero_nyquist(p, w.A, batch * p.nN, st)));
  if (!p.wigner) return fr.run(p.fft_phi, w.A, f, plane, CUFFT_INVERSE);
  S2GB_TRY(fr.run(p.fft_phi, w.A, w.B, (size_t)p.nN * plane, CUFFT_INVERSE));
  S2GB_TRY(cuda_rc(launch_gamma_reorder(p, w.B, w.C, batch, 0, 1.0, st)));
  return gamma_dft(p, w.C, f, batch, w.fft, st, CUFFT_INVERSE);
}

int do_adjoint_inverse(Plan& p, const void* fbar, void* flmbar, int batch, const Workspace& w,
                       cudaStream_t st) {
  FftRunner fr{p, st, w.fft, batch};
  const size_t plane = (size_t)p.R * p.P;
  const void* sig_in = fbar;
  if (p.wigner) {
    S2GB_TRY(gamma_dft(p, fbar, w.C, batch, w.fft, st, CUFFT_FORWARD));
    S2GB_TRY(cuda_rc(launch_gamma_reorder(p, w.C, w.B, batch, 1, 1.0, st)));
    sig_in = w.B;
  }
  S2GB_TRY(fr.run(p.fft_phi, sig_in, w.A, (size_t)p.nN * plane, CUFFT_FORWARD));
  FwdArgs a = fwd_args(p, w.A, flmbar, batch, p.scale_inv, (long long)plane, p.P, 1, 1, 0);
  a.part = w.D;
  a.mpart = w.D;
  return cuda_rc(launch_theta_forward(p, a, st));
}

int do_adjoint_forward(Plan& p, const void* flmbar, void* fbar, int batch, const Workspace& w,
                       cudaStream_t st) {
  FftRunner fr{p, st, w.fft, batch};
  const int S = batch * p.nN;
  const size_t plane = (size_t)p.R * p.P;
  if (p.sampling == S2GB_DH) {
    InvArgs a = inv_args(p, flmbar, w.A, batch, p.scale_fwd, (long long)plane, p.P, 1, 1);
    a.mpart = w.D;
    S2GB_TRY(cuda_rc(launch_theta_inverse(p, a, st)));
    S2GB_TRY(cuda_rc(launch_ring_weight(p, w.A, S, p.P, st)));
  } else {
    InvArgs a = inv_args(p, flmbar, w.B, batch, p.scale_fwd, (long long)p.MR * p.TS, 1, p.TS, 0);
    a.mpart = w.D;
    S2GB_TRY(cuda_rc(launch_theta_inverse(p, a, st)));
    S2GB_TRY(cuda_rc(launch_nu_extend(p, w.B, S * p.MR, st)));
    S2GB_TRY(theta_weight_operator(p, fr, w.A, w.B, S));
    S2GB_TRY(cuda_rc(launch_extend_adjoint(p, w.B, w.A, S, st)));
  }
  if (!p.wigner) return fr.run(p.fft_phi, w.A, fbar, plane, CUFFT_INVERSE);
  S2GB_TRY(fr.run(p.fft_phi, w.A, w.B, (size_t)p.nN * plane, CUFFT_INVERSE));
  S2GB_TRY(cuda_rc(launch_gamma_reorder(p, w.B, w.C, batch, 0, kTwoPi / (2 * p.N - 1), st)));
  return gamma_dft(p, w.C, fbar, batch, w.fft, st, CUFFT_INVERSE);
}

// ---- real signals (spin 0, Sec. 2.2 Hermitian symmetry flm(l, -m) = (-1)^m conj(flm(l, m))) ----
// f real [b][R][P]; flm [b][L][L] holds the orders m = 0..L-1; ring spectra [b][t][m] with L
// columns.  Every stage runs on the orders m >= 0 only; the phi DFTs are real-to-complex and
// complex-to-real (the C2R sum is Re X_0 + 2 Re sum_{m>=1} X_m e^{i m phi}).  MW and DH (P = 2L-1).

int do_forward_real(Plan& p, const void* f, void* flm, int batch, const Workspace& w, cudaStream_t st,
                    int mlo, int mhi) {
  FftRunner fr{p, st, w.fft, batch};
  const size_t L = p.L, R = p.R, P = p.P, TS = p.TS;
  S2GB_TRY(fr.run_real(p.fft_phi, f, w.A, R * P, R * L, +1));
  FwdArgs a;
  if (p.sampling == S2GB_DH) {
    a = fwd_args(p, w.A, flm, batch, p.scale_fwd, (long long)(R * L), (long long)L, 1, 1, 1);
  } else {
    if (p.tc_op) {
      S2GB_TRY(cuda_rc(launch_operator_tc(p, w.A, w.B, operator_cexp(p, w, batch, L), batch, st)));
    } else {
      S2GB_TRY(cuda_rc(launch_extend(p, w.A, w.B, batch, st)));
      S2GB_TRY(theta_weight_operator(p, fr, w.A, w.B, batch));
    }
    a = fwd_args(p, w.B, flm, batch, p.scale_fwd, (long long)(L * TS), 1, (long long)TS, 1, 1);
  }
  a.part = w.D;
  order_ranks(p, mlo, mhi, a.rank0, a.nrank);
  return cuda_rc(launch_theta_forward(p, a, st));
}

int do_inverse_real(Plan& p, const void* flm, void* f, int batch, const Workspace& w, cudaStream_t st) {
  FftRunner fr{p, st, w.fft, batch};
  const size_t L = p.L, R = p.R, P = p.P;
  InvArgs a = inv_args(p, flm, w.A, batch, p.scale_inv, (long long)(R * L), (long long)L, 1, 1);
  S2GB_TRY(cuda_rc(launch_theta_inverse(p, a, st)));
  return fr.run_real(p.fft_phi_c2r, w.A, f, R * L, R * P, -1);
}

// Adjoint (real inner product) of f = C2R(theta(flm)): R2C, columns m >= 1 doubled, then the
// forward-shaped theta contraction without weights.
int do_adjoint_inverse_real(Plan& p, const void* fbar, void* flmbar, int batch, const Workspace& w,
                            cudaStream_t st) {
  FftRunner fr{p, st, w.fft, batch};
  const size_t L = p.L, R = p.R, P = p.P;
  S2GB_TRY(fr.run_real(p.fft_phi, fbar, w.A, R * P, R * L, +1));
  S2GB_TRY(cuda_rc(launch_scale_nonzero_orders(p, w.A, (size_t)batch * R, 2.0, st)));
  FwdArgs a = fwd_args(p, w.A, flmbar, batch, p.scale_inv, (long long)(R * L), (long long)L, 1, 1, 0);
  a.part = w.D;
  return cuda_rc(launch_theta_forward(p, a, st));
}

// Adjoint of the real forward: the complex adjoint's stages on the orders m >= 0, then the
// adjoint of R2C, which is C2R of the spectrum with columns m >= 1 halved (and Im X_0 dropped).
int do_adjoint_forward_real(Plan& p, const void* flmbar, void* fbar, int batch, const Workspace& w,
                            cudaStream_t st) {
  FftRunner fr{p, st, w.fft, batch};
  const size_t L = p.L, R = p.R, P = p.P, TS = p.TS;
  if (p.sampling == S2GB_DH) {
    InvArgs a = inv_args(p, flmbar, w.A, batch, p.scale_fwd, (long long)(R * L), (long long)L, 1, 1);
    S2GB_TRY(cuda_rc(launch_theta_inverse(p, a, st)));
    S2GB_TRY(cuda_rc(launch_ring_weight(p, w.A, batch, (int)L, st)));
  } else {
    InvArgs a = inv_args(p, flmbar, w.B, batch, p.scale_fwd, (long long)(L * TS), 1, (long long)TS, 1);
    S2GB_TRY(cuda_rc(launch_theta_inverse(p, a, st)));
    S2GB_TRY(cuda_rc(launch_nu_extend(p, w.B, batch * p.MR, st)));
    S2GB_TRY(theta_weight_operator(p, fr, w.A, w.B, batch));
    S2GB_TRY(cuda_rc(launch_extend_adjoint(p, w.B, w.A, batch, st)));
  }
  S2GB_TRY(cuda_rc(launch_scale_nonzero_orders(p, w.A, (size_t)batch * R, 0.5, st)));
  return fr.run_real(p.fft_phi_c2r, w.A, fbar, R * L, R * P, -1);
}

int do_inverse_phi_real(Plan& p, const void* ftilde, void* f, int batch, const Workspace& w, cudaStream_t st) {
  FftRunner fr{p, st, w.fft, batch};
  return fr.run_real(p.fft_phi_c2r, ftilde, f, (size_t)p.R * p.L, (size_t)p.R * p.P, -1);
}

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bbytes && y < x + abytes;
}

enum class Op { Forward, Inverse, AdjForward, AdjInverse, InversePhi };

int run(s2gb_plan plan, Op op, const void* in, void* out, int batch, void* ws, size_t ws_bytes,
        void* stream, int mlo = 0, int mhi = -1) {
  if (!plan || !in || !out) return S2GB_EINVAL;
  Plan& p = plan->p;
  if (batch < 1 || batch > p.max_batch) return S2GB_EINVAL;
  if (mhi < 0) mhi = p.L;
  if (mlo < 0 || mlo > mhi || mhi > p.L) return S2GB_EINVAL;
  if (op == Op::InversePhi && p.wigner) return S2GB_EUNSUPPORTED;
  const size_t es = p.precision == S2GB_FP64 ? 16 : 8;
  // bytes of the signal side and of the coefficient side (ring spectra for InversePhi)
  const size_t sig_bytes = (size_t)batch * p.nN * p.R * p.P * (p.real ? es / 2 : es);
  const size_t coef_bytes = op == Op::InversePhi ? (size_t)batch * p.R * (p.real ? p.L : p.P) * es
                                                 : (size_t)batch * p.nN * p.L * p.MR * es;
  const bool in_is_signal = (op == Op::Forward || op == Op::AdjInverse);
  if (overlaps(in, in_is_signal ? sig_bytes : coef_bytes, out, in_is_signal ? coef_bytes : sig_bytes))
    return S2GB_EINVAL;
  if (!ws || ws_bytes < workspace_bytes(p, batch)) return S2GB_EWORKSPACE;
  DeviceGuard g(p.device);
  std::lock_guard<std::mutex> lock(p.fft_mutex);
  const Workspace w = carve(p, ws, batch);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (p.real) {
    switch (op) {
      case Op::Forward: return do_forward_real(p, in, out, batch, w, st, mlo, mhi);
      case Op::InversePhi: return do_inverse_phi_real(p, in, out, batch, w, st);
      case Op::Inverse: return do_inverse_real(p, in, out, batch, w, st);
      case Op::AdjForward: return do_adjoint_forward_real(p, in, out, batch, w, st);
      case Op::AdjInverse: return do_adjoint_inverse_real(p, in, out, batch, w, st);
    }
    return S2GB_EINVAL;
  }
  switch (op) {
    case Op::Forward: return do_forward(p, in, out, batch, w, st, mlo, mhi);
    case Op::InversePhi: return do_inverse_phi(p, in, out, batch, w, st);
    case Op::Inverse: return do_inverse(p, in, out, batch, w, st);
    case Op::AdjForward: return do_adjoint_forward(p, in, out, batch, w, st);
    case Op::AdjInverse: return do_adjoint_inverse(p, in, out, batch, w, st);
  }
  return S2GB_EINVAL;
}

}  // namespace
}  // namespace s2gb

using s2gb::Op;

extern "C" {

namespace {
int plan_create_impl(s2gb_plan* out, int L, int spin, int N, int sampling, int precision, int max_batch,
                     int device, bool real, bool precompute = false, bool mrec = false,
                     bool fma_contraction = false) {
  if (!out) return S2GB_EINVAL;
  *out = nullptr;
  if (L < 1 || L > 8192 || N < 0 || N > L || max_batch < 1) return S2GB_EINVAL;
  if (sampling != S2GB_MW && sampling != S2GB_MWSS && sampling != S2GB_DH) return S2GB_EINVAL;
  if (precision != S2GB_FP64 && precision != S2GB_FP32) return S2GB_EINVAL;
  if (N == 0 && (spin <= -L || spin >= L)) return S2GB_EINVAL;
  // rings of the recursion kernels (MWSS: the interior; its two pole rings are handled exactly)
  const int rings = sampling == S2GB_MWSS ? L - 1 : (sampling == S2GB_DH ? 2 * L : L);
  // float32 forward kernels hold every ring in one CTA; the ring-chunked float64 forward keeps its
  // polar caps (under 0.05 of the rings each) within one 512-ring launch, i.e. at most 8192 rings
  if (precision == S2GB_FP32 && (L > 2048 || rings > s2gb::kFwdChunk)) return S2GB_EUNSUPPORTED;
  if (rings > 8192) return S2GB_EUNSUPPORTED;
  if (real && sampling == S2GB_MWSS) return S2GB_EUNSUPPORTED;
  if (precompute && (precision != S2GB_FP64 || L > s2gb::kFwdChunk || sampling != S2GB_MW))
    return S2GB_EUNSUPPORTED;
  if (mrec && (precision != S2GB_FP64 || real || precompute)) return S2GB_EUNSUPPORTED;
  {
    // the cuFFT plans take 32-bit batch counts: max_batch * (2N-1) signals times the rows of the
    // largest batched FFT (the rings of the phi DFT, or the order rows of the theta operator)
    const long long nsig = (long long)max_batch * (N >= 1 ? 2LL * N - 1 : 1LL);
    const long long rings_all = sampling == S2GB_DH ? 2LL * L : (sampling == S2GB_MWSS ? L + 1LL : (long long)L);
    const long long order_rows = real ? (long long)L : 2LL * L - 1;
    if (nsig * (rings_all > order_rows ? rings_all : order_rows) > 2147483647LL) return S2GB_EUNSUPPORTED;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return S2GB_EINVAL;
  s2gb_plan h = new (std::nothrow) s2gb_plan_s;
  if (!h) return S2GB_ENOMEM;
  s2gb::Plan& p = h->p;
  p.L = L; p.spin = N == 0 ? spin : 0; p.N = N; p.precision = precision; p.max_batch = max_batch;
  p.device = device;
  p.sampling = sampling;
  p.real = real;
  p.precompute = precompute;
  p.mrec = mrec;
  p.tc = precision == S2GB_FP64 && !precompute && !mrec && !fma_contraction;
  // float32: the tensor-core inverse pays off from 16 signals per call (measured on GB300)
  p.tc32 = precision == S2GB_FP32 && !fma_contraction && max_batch >= 16;
  int rc;
  {
    s2gb::DeviceGuard g(device);
    rc = s2gb::make_plan(&p);
    if (rc == S2GB_OK) rc = s2gb::build_theta_operator(p);
    if (rc != S2GB_OK) s2gb::free_plan(&p);
  }
  if (rc != S2GB_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return S2GB_OK;
}

}  // namespace

int s2gb_plan_create(s2gb_plan* out, int L, int spin, int N, int sampling, int precision,
                     int max_batch, int device) {
  return plan_create_impl(out, L, spin, N, sampling, precision, max_batch, device, false);
}

int s2gb_plan_create_real(s2gb_plan* out, int L, int sampling, int precision, int max_batch, int device) {
  return plan_create_impl(out, L, 0, 0, sampling, precision, max_batch, device, true);
}

int s2gb_plan_create_flags(s2gb_plan* out, int L, int spin, int N, int sampling, int precision,
                           int max_batch, int device, unsigned flags) {
  if (out) *out = nullptr;
  if (flags & ~(unsigned)(S2GB_PLAN_REAL | S2GB_PLAN_PRECOMPUTE | S2GB_PLAN_MRECURSION |
                          S2GB_PLAN_FMA_CONTRACTION))
    return S2GB_EINVAL;
  const bool real = (flags & S2GB_PLAN_REAL) != 0;
  if (real && (spin != 0 || N != 0)) return S2GB_EINVAL;
  return plan_create_impl(out, L, spin, N, sampling, precision, max_batch, device, real,
                          (flags & S2GB_PLAN_PRECOMPUTE) != 0, (flags & S2GB_PLAN_MRECURSION) != 0,
                          (flags & S2GB_PLAN_FMA_CONTRACTION) != 0);
}

void s2gb_plan_destroy(s2gb_plan plan) {
  if (!plan) return;
  {
    s2gb::DeviceGuard g(plan->p.device);
    s2gb::free_plan(&plan->p);
  }
  delete plan;
}

size_t s2gb_workspace_bytes(s2gb_plan plan, int batch) {
  if (!plan) return 0;
  return s2gb::workspace_bytes(plan->p, batch);
}

size_t s2gb_plan_device_bytes(s2gb_plan plan) { return plan ? plan->p.device_bytes : 0; }

int s2gb_forward(s2gb_plan plan, const void* f, void* flm, int batch, void* ws, size_t ws_bytes, void* stream) {
  return s2gb::run(plan, Op::Forward, f, flm, batch, ws, ws_bytes, stream);
}
int s2gb_inverse(s2gb_plan plan, const void* flm, void* f, int batch, void* ws, size_t ws_bytes, void* stream) {
  return s2gb::run(plan, Op::Inverse, flm, f, batch, ws, ws_bytes, stream);
}
int s2gb_adjoint_forward(s2gb_plan plan, const void* flm_bar, void* f_bar, int batch, void* ws,
                         size_t ws_bytes, void* stream) {
  return s2gb::run(plan, Op::AdjForward, flm_bar, f_bar, batch, ws, ws_bytes, stream);
}
int s2gb_adjoint_inverse(s2gb_plan plan, const void* f_bar, void* flm_bar, int batch, void* ws,
                         size_t ws_bytes, void* stream) {
  return s2gb::run(plan, Op::AdjInverse, f_bar, flm_bar, batch, ws, ws_bytes, stream);
}

int s2gb_inverse_theta_mrange(s2gb_plan plan, const void* flm, void* ftilde, int batch, int m_lo,
                              int m_hi, void* stream) {
  if (!plan || !flm || !ftilde) return S2GB_EINVAL;
  s2gb::Plan& p = plan->p;
  if (p.wigner || p.mrec) return S2GB_EUNSUPPORTED;   // order recursion: its partials need a workspace
  if (batch < 1 || batch > p.max_batch) return S2GB_EINVAL;
  if (m_lo < 0 || m_lo > m_hi || m_hi > p.L) return S2GB_EINVAL;
  const size_t es = p.precision == S2GB_FP64 ? 16 : 8;
  const int SW = p.real ? p.L : p.P;     // ring-spectrum columns
  if (s2gb::overlaps(flm, (size_t)batch * p.L * p.MR * es, ftilde, (size_t)batch * p.R * SW * es))
    return S2GB_EINVAL;
  s2gb::DeviceGuard g(p.device);
  s2gb::InvArgs a = s2gb::inv_args(p, flm, ftilde, batch, p.scale_inv, (long long)p.R * SW, SW, 1, 1);
  s2gb::order_ranks(p, m_lo, m_hi, a.rank0, a.nrank);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = s2gb::cuda_rc(s2gb::launch_theta_inverse(p, a, st));
  if (rc != S2GB_OK) return rc;
  return s2gb::cuda_rc(s2gb::zero_nyquist(p, ftilde, batch, st));
}

int s2gb_inverse_theta(s2gb_plan plan, const void* flm, void* ftilde, int batch, void* stream) {
  return s2gb_inverse_theta_mrange(plan, flm, ftilde, batch, 0, plan ? plan->p.L : 0, stream);
}

int s2gb_forward_mrange(s2gb_plan plan, const void* f, void* flm, int batch, int m_lo, int m_hi,
                        void* ws, size_t ws_bytes, void* stream) {
  return s2gb::run(plan, Op::Forward, f, flm, batch, ws, ws_bytes, stream, m_lo, m_hi);
}

int s2gb_inverse_phi(s2gb_plan plan, const void* ftilde, void* f, int batch, void* ws, size_t ws_bytes,
                     void* stream) {
  return s2gb::run(plan, Op::InversePhi, ftilde, f, batch, ws, ws_bytes, stream);
}

int s2gb_forward_theta(s2gb_plan plan, const void* gin, void* flm, int batch, void* stream) {
  if (!plan || !gin || !flm) return S2GB_EINVAL;
  s2gb::Plan& p = plan->p;
  if (p.wigner || p.fwd_parts > 1 || p.mrec) return S2GB_EUNSUPPORTED;   // these need a workspace
  if (batch < 1 || batch > p.max_batch) return S2GB_EINVAL;
  const size_t es = p.precision == S2GB_FP64 ? 16 : 8;
  if (s2gb::overlaps(gin, (size_t)batch * p.MR * p.R * es, flm, (size_t)batch * p.L * p.MR * es))
    return S2GB_EINVAL;
  s2gb::DeviceGuard g(p.device);
  s2gb::FwdArgs a = s2gb::fwd_args(p, gin, flm, batch, p.scale_fwd, (long long)p.MR * p.R, 1, p.R,
                                   p.real ? 1 : 0, 0);
  return s2gb::cuda_rc(s2gb::launch_theta_forward(p, a, reinterpret_cast<cudaStream_t>(stream)));
}

unsigned long long s2gb_kernels_launched(void) {
  return s2gb::g_kernel_launches.load(std::memory_order_relaxed);
}

const char* s2gb_strerror(int code) {
  switch (code) {
    case S2GB_OK: return "success";
    case S2GB_EINVAL: return "invalid argument";
    case S2GB_EUNSUPPORTED: return "unsupported configuration";
    case S2GB_ENOMEM: return "device allocation failed";
    case S2GB_ECUDA: return "CUDA runtime error";
    case S2GB_ECUFFT: return "cuFFT error";
    case S2GB_EWORKSPACE: return "workspace missing or too small";
    default: return "unknown error code";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Allocation-free inverse transform (s2gb_inverse_noalloc).
//
// Its scratch is this file-scope device array instead of a caller-provided workspace.  Every
// device that loads the library holds the array until the process exits.  Host code cannot pass
// the symbol itself to a kernel (on the host it names a stand-in, not device memory), so the
// device address is looked up with cudaGetSymbolAddress, once per device, with that device
// current, the first time the entry point runs there.
// ---------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char s2gb_noalloc_scratch[S2GB_NOALLOC_SCRATCH_BYTES];

namespace s2gb {
namespace {

std::mutex g_noalloc_mutex;
constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (device < 0 || device >= kMaxDevices) return S2GB_EINVAL;
  if (!g_noalloc_ptr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, s2gb_noalloc_scratch) != cudaSuccess || !ptr) return S2GB_ECUDA;
    g_noalloc_ptr[device] = ptr;
  }
  *out = g_noalloc_ptr[device];
  return S2GB_OK;
}

}  // namespace
}  // namespace s2gb

extern "C" int s2gb_inverse_noalloc(s2gb_plan plan, const void* flm, void* f, int batch, void* stream) {
  if (!plan || !flm || !f) return S2GB_EINVAL;
  s2gb::Plan& p = plan->p;
  if (p.real || p.mrec) return S2GB_EUNSUPPORTED;
  if (batch < 1 || batch > p.max_batch) return S2GB_EINVAL;
  const size_t es = p.precision == S2GB_FP64 ? 16 : 8;
  const size_t sig_bytes = (size_t)batch * p.nN * p.R * p.P * es;
  if (s2gb::overlaps(flm, (size_t)batch * p.nN * p.L * p.T * es, f, sig_bytes)) return S2GB_EINVAL;
  // scratch: the theta-stage output (and, for Wigner, two more signal-sized buffers) + cuFFT work
  const int q = (batch == p.max_batch) ? 1 : 0;
  size_t work = 0, w2 = 0;
  if (cufftGetSize(p.fft_phi[q], &work) != CUFFT_SUCCESS) return S2GB_ECUFFT;
  if (p.wigner) {
    if (cufftGetSize(p.fft_gam[0], &w2) != CUFFT_SUCCESS) return S2GB_ECUFFT;
    if (w2 > work) work = w2;
  }
  const size_t buf = s2gb::align256(sig_bytes);
  const int nbuf = p.wigner ? 3 : 1;
  const size_t need = nbuf * buf + s2gb::align256(work);
  if (need > (size_t)S2GB_NOALLOC_SCRATCH_BYTES) return S2GB_EWORKSPACE;
  s2gb::DeviceGuard g(p.device);
  void* base = nullptr;
  int rc = s2gb::noalloc_scratch(p.device, &base);
  if (rc != S2GB_OK) return rc;
  char* b = reinterpret_cast<char*>(base);
  s2gb::Workspace w = {b, b + (nbuf > 1 ? buf : 0), b + (nbuf > 2 ? 2 * buf : 0), b + nbuf * buf};
  std::lock_guard<std::mutex> lock(p.fft_mutex);
  return s2gb::do_inverse(p, flm, f, batch, w, reinterpret_cast<cudaStream_t>(stream));
}
