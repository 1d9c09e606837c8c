// Plan creation: host-side tables in extended precision, the recursion-coefficient kernel in
// double-double arithmetic, FFT weights and cuFFT plans.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <vector>

#include "dd.cuh"
#include "s2gb_internal.h"

namespace s2gb {

namespace {

constexpr long double kPiL = 3.141592653589793238462643383279502884197169399375105820974944L;
constexpr double kPi = 3.14159265358979323846;

// log2(k!) for k = 0..kmax, compensated running sum in long double.
std::vector<long double> log2_factorials(int kmax) {
  std::vector<long double> out(kmax + 1, 0.0L);
  long double s = 0.0L, c = 0.0L;
  for (int k = 1; k <= kmax; ++k) {
    long double x = std::log2((long double)k);
    long double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
    out[k] = s + c;
  }
  return out;
}

void split(long double v, double* hi, double* lo) {
  double h = (double)v;
  *hi = h;
  *lo = std::isfinite(h) ? (double)(v - (long double)h) : 0.0;
}

// Recursion coefficients of the step j -> j+1 for every (n, m, j), in double-double, then rounded.
//   d^{j+1} = A_j (cos t - B_j) d^j - C_j d^{j-1}
//   A_j = (2j+1)(j+1) / sqrt(((j+1)^2-m^2)((j+1)^2-n^2)),  B_j = m n / (j (j+1)),
//   C_j = (j+1) sqrt((j^2-m^2)(j^2-n^2)) / (j sqrt(((j+1)^2-m^2)((j+1)^2-n^2)))
// (the three-term recurrence of the Wigner d-functions in the degree, obtained from the Jacobi
// representation of Sec. 3.1 through the Jacobi polynomials' own three-term recurrence).
// Stored per step: A, C, K_n = A(1-B), K_s = -A(1+B), Kd_n = K_n - 1 - C, Kd_s = K_s + 1 + C.
// The Kd are differences of O(1) terms that nearly cancel for j >> |m|,|n|; evaluating them in
// double-double keeps them accurate to a few ulps of their own size.
__global__ void coef_kernel(double* coef, const int* n_of, int nN, int L) {
  const int T = 2 * L - 1;
  long long total = (long long)nN * T * L;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % L);
    const int mi = (int)((idx / L) % T);
    const int ni = (int)(idx / ((long long)L * T));
    const long long m = mi - (L - 1);
    const long long n = n_of[ni];
    double* out = coef + idx * kCoefPerStep;
    const long long l0 = (m < 0 ? -m : m) > (n < 0 ? -n : n) ? (m < 0 ? -m : m) : (n < 0 ? -n : n);
    if (j < l0 || j >= L - 1) {
      for (int q = 0; q < kCoefPerStep; ++q) out[q] = 0.0;
      continue;
    }
    const long long j1 = j + 1;
    const long long X1 = (j1 * j1 - m * m) * (j1 * j1 - n * n);
    const long long X0 = ((long long)j * j - m * m) * ((long long)j * j - n * n);
    dd R1 = dd_sqrt(dd_from_ll(X1));
    dd R0 = dd_sqrt(dd_from_ll(X0));
    dd A = dd_div(dd_from_ll((2LL * j + 1) * j1), R1);
    dd B = {0.0, 0.0}, C = {0.0, 0.0};
    if (j > 0) {
      B = dd_div(dd_from_ll(m * n), dd_from_ll((long long)j * j1));
      C = dd_div(dd_mul(dd_from_ll(j1), R0), dd_mul(dd_from_ll(j), R1));
    }
    dd one = {1.0, 0.0};
    dd Kn = dd_mul(A, dd_sub(one, B));
    dd Ks = dd_neg(dd_mul(A, dd_add(one, B)));
    dd Kdn = dd_sub(dd_sub(Kn, one), C);
    dd Kds = dd_add(dd_add(Ks, one), C);
    out[0] = A.hi + A.lo;
    out[1] = C.hi + C.lo;
    out[2] = Kn.hi + Kn.lo;
    out[3] = Ks.hi + Ks.lo;
    out[4] = Kdn.hi + Kdn.lo;
    out[5] = Kds.hi + Kds.lo;
  }
}

// Normalised coefficients for the float64 kernels.  Along the chain of an order, from l0 =
// max(|m|, |n|), the plain recurrence is carried for u^j = d^j / gamma_j with
//   gamma_{l0-1} = gamma_{l0} = 1,  gamma_{j+1} = C_j gamma_{j-1}  (= 1 where C_j = 0, i.e. j = l0),
// which turns d^{j+1} = P_j d^j - C_j d^{j-1} into u^{j+1} = (P_j gamma_j/gamma_{j+1}) u^j - u^{j-1}
// (2 FMA per step instead of 3).  The difference form carries e^j = eta_j ehat^j with
//   eta_{l0} = 1,  eta_{j+1} = C_j eta_j  (= 1 where C_j = 0),
// so ehat^{j+1} = (Q_j / eta_{j+1}) d^j + sigma ehat^j and d^{j+1} = sigma d^j + eta_{j+1} ehat^{j+1}.
// The kernels never convert back: the contraction takes gamma_j into the coefficient (inverse) or
// the output scale (forward).  C_k = (k+1) sqrt((k^2-m^2)(k^2-n^2)) / (k sqrt(((k+1)^2-m^2)((k+1)^2-n^2)))
// telescopes, so the products stay close to 1: gamma in [2^-7, 1] and eta in [2^-13, 1] for every
// order up to L = 8192.
__device__ void coef_terms(long long j, long long m, long long n, dd& A, dd& B, dd& C) {
  const long long j1 = j + 1;
  const long long X1 = (j1 * j1 - m * m) * (j1 * j1 - n * n);
  const long long X0 = (j * j - m * m) * (j * j - n * n);
  dd R1 = dd_sqrt(dd_from_ll(X1));
  dd R0 = dd_sqrt(dd_from_ll(X0));
  A = dd_div(dd_from_ll((2LL * j + 1) * j1), R1);
  B = {0.0, 0.0};
  C = {0.0, 0.0};
  if (j > 0) {
    B = dd_div(dd_from_ll(m * n), dd_from_ll(j * j1));
    C = dd_div(dd_mul(dd_from_ll(j1), R0), dd_mul(dd_from_ll(j), R1));
  }
}

// One thread per (n, m): the chain's steps in order, the products gamma and eta carried in
// double-double and every table entry rounded once.
__global__ void coefn_kernel(double* coef, const int* n_of, int nN, int L) {
  const int T = 2 * L - 1;
  const long long total = (long long)nN * T;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int mi = (int)(idx % T);
    const int ni = (int)(idx / T);
    const long long m = mi - (L - 1);
    const long long n = n_of[ni];
    double* out = coef + idx * (long long)L * kCoefPerStepN;
    const long long am = m < 0 ? -m : m, an = n < 0 ? -n : n;
    const long long l0 = am > an ? am : an;
    const dd one = {1.0, 0.0};
    dd g_prev = one, g_cur = one, e_cur = one;     // gamma_{j-1}, gamma_j, eta_j
    for (long long j = 0; j < L; ++j, out += kCoefPerStepN) {
      if (j < l0) {
        for (int q = 0; q < kCoefPerStepN; ++q) out[q] = 0.0;
        continue;
      }
      dd A, B, C;
      coef_terms(j, m, n, A, B, C);
      const bool cz = (C.hi == 0.0);
      const dd g_next = cz ? one : dd_mul(C, g_prev);   // gamma_{j+1}
      const dd e_next = cz ? one : dd_mul(C, e_cur);    // eta_{j+1}
      const dd r = dd_div(g_cur, g_next);
      const dd Kn = dd_mul(A, dd_sub(one, B));
      const dd Ks = dd_neg(dd_mul(A, dd_add(one, B)));
      const dd Kdn = dd_sub(dd_sub(Kn, one), C);
      const dd Kds = dd_add(dd_add(Ks, one), C);
      const dd Ap = dd_mul(A, r), Knp = dd_mul(Kn, r), Ksp = dd_mul(Ks, r);
      const dd App = dd_div(A, e_next), Kdnp = dd_div(Kdn, e_next), Kdsp = dd_div(Kds, e_next);
      const dd ig = dd_div(one, g_cur);
      out[0] = Ap.hi + Ap.lo;
      out[1] = Knp.hi + Knp.lo;
      out[2] = Ksp.hi + Ksp.lo;
      out[3] = g_cur.hi + g_cur.lo;
      out[4] = g_next.hi + g_next.lo;
      out[5] = App.hi + App.lo;
      out[6] = Kdnp.hi + Kdnp.lo;
      out[7] = Kdsp.hi + Kdsp.lo;
      out[8] = e_next.hi + e_next.lo;
      out[9] = ig.hi + ig.lo;
      g_prev = g_cur;
      g_cur = g_next;
      e_cur = e_next;
    }
  }
}

// Coefficients of the order recursion (Sec. 3.3, Eq. "wigner-d-recursion") for the step m -> m-1
// at degree l: (A, B) = (a_{m-1}, a_{m-1}/a_m), a_m = 2/sqrt((l-m)(l+m+1)), for -l < m <= l
// (B = 0 at m = l, where d_{l+1} = 0), in double-double and rounded once.  Layout [l][m + L - 1].
__global__ void mrec_ab_kernel(double* ab, int L) {
  const int T = 2 * L - 1;
  const long long total = (long long)L * T;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long l = idx / T;
    const long long m = idx % T - (L - 1);
    double* out = ab + 2 * idx;
    if (m > l || m <= -l) {
      out[0] = 0.0; out[1] = 0.0;
      continue;
    }
    const dd R1 = dd_sqrt(dd_from_ll((l - m + 1) * (l + m)));
    const dd A = dd_div(dd_from_ll(2), R1);
    const dd B = (m == l) ? dd{0.0, 0.0} : dd_div(dd_sqrt(dd_from_ll((l - m) * (l + m + 1))), R1);
    out[0] = A.hi + A.lo;
    out[1] = B.hi + B.lo;
  }
}

__global__ void to_float_kernel(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

int good_fft_size(int n) {
  // smallest m >= n whose prime factors are in {2, 3, 5, 7}
  for (int m = n > 1 ? n : 1;; ++m) {
    int r = m;
    for (int p : {2, 3, 5, 7})
      while (r % p == 0) r /= p;
    if (r == 1) return m;
  }
}

template <typename T>
int upload(T** dst, const std::vector<T>& src, size_t* counter) {
  size_t bytes = src.size() * sizeof(T);
  if (cudaMalloc((void**)dst, bytes > 0 ? bytes : sizeof(T)) != cudaSuccess) return S2GB_ENOMEM;
  *counter += bytes;
  if (bytes && cudaMemcpy(*dst, src.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) return S2GB_ECUDA;
  return S2GB_OK;
}

int make_fft(cufftHandle* h, int n, int batch, int istride, int idist, cufftType type, size_t* work,
             int odist = 0) {
  if (cufftCreate(h) != CUFFT_SUCCESS) return S2GB_ECUFFT;
  if (cufftSetAutoAllocation(*h, 0) != CUFFT_SUCCESS) return S2GB_ECUFFT;
  int nn[1] = {n};
  int emb[1] = {n};
  size_t ws = 0;
  cufftResult r = cufftMakePlanMany(*h, 1, nn, emb, istride, idist, emb, istride, odist ? odist : idist,
                                    type, batch, &ws);
  if (r != CUFFT_SUCCESS) return S2GB_ECUFFT;
  if (ws > *work) *work = ws;
  return S2GB_OK;
}

// DH theta weights (Sec. 4.2.1) times the phi step 2 pi / P: q_t = (2/L) sin(theta_t)
// sum_{k<L} sin((2k+1) theta_t) / (2k+1) with theta_t = (2t+1) pi / (4L).  Every sine has its
// argument reduced exactly ((2k+1)(2t+1) mod 8L, in units of pi/(4L)) and the sum is compensated
// (Neumaier), so each weight is accurate to a few ulps.  q_{2L-1-t} = q_t (theta -> pi - theta).
std::vector<double> dh_ring_weights(int L) {
  std::vector<double> q(2 * L);
  const long long M = 8LL * L;
  const double u = kPi / (4.0 * L);
  for (int t = 0; t < L; ++t) {
    double s = 0.0, c = 0.0;
    for (int k = 0; k < L; ++k) {
      const long long num = ((2LL * k + 1) * (2LL * t + 1)) % M;
      const double x = std::sin((double)num * u) / (double)(2 * k + 1);
      const double ts = s + x;
      c += std::fabs(s) >= std::fabs(x) ? (s - ts) + x : (x - ts) + s;
      s = ts;
    }
    const long double th = (long double)(2 * t + 1) * kPiL / (4.0L * L);
    const long double w = (2.0L / L) * std::sin(th) * ((long double)s + (long double)c);
    q[t] = q[2 * L - 1 - t] = (double)(w * 2.0L * kPiL / (long double)(2 * L - 1));
  }
  return q;
}

}  // namespace

int make_plan(Plan* p) {
  const int L = p->L;
  const int T = 2 * L - 1;
  p->T = T;
  p->wigner = p->N >= 1;
  p->nN = p->wigner ? 2 * p->N - 1 : 1;
  p->MR = p->real ? L : T;
  switch (p->sampling) {
    case S2GB_MWSS: p->R = L + 1; p->P = 2 * L; p->TS = 2 * L; break;
    case S2GB_DH: p->R = 2 * L; p->P = T; p->TS = 0; break;
    default: p->R = L; p->P = T; p->TS = T; break;
  }
  p->Nfft = p->TS ? good_fft_size(4 * L - 3 > p->TS ? 4 * L - 3 : p->TS) : 0;
  const int nN = p->nN;
  const int R = p->R;

  std::vector<int> n_of(nN);
  for (int i = 0; i < nN; ++i) n_of[i] = p->wigner ? i - (p->N - 1) : -p->spin;

  // ---- rings (Sec. 4.2) ----
  // MW: theta_t = (2t+1) pi/(2L-1), t < L (the last ring is theta = pi);
  // MWSS: theta_t = pi t/L, t <= L (theta = 0 and pi are rings); DH: theta_t = (2t+1) pi/(4L), t < 2L.
  std::vector<RingData> ring(R);
  for (int t = 0; t < R; ++t) {
    RingData r{};
    int pole = 0;
    long double th;
    if (p->sampling == S2GB_MWSS) {
      pole = (t == L) ? 1 : (t == 0 ? 2 : 0);
      th = pole == 1 ? kPiL : (long double)t * kPiL / (long double)L;
    } else if (p->sampling == S2GB_DH) {
      th = (long double)(2 * t + 1) * kPiL / (4.0L * L);
    } else {
      pole = (t == L - 1) ? 1 : 0;
      th = pole ? kPiL : (long double)(2 * t + 1) * kPiL / (long double)T;
    }
    long double sh = pole == 2 ? 0.0L : std::sin(th / 2), ch = pole == 1 ? 0.0L : std::cos(th / 2);
    r.north = th < kPiL / 2;
    r.pole = pole;
    r.v = (double)(r.north ? 2 * sh * sh : 2 * ch * ch);
    if (pole == 2) {
      r.ls_hi = -std::numeric_limits<double>::infinity();
      r.ls_lo = 0.0;
    } else {
      split(std::log2(sh), &r.ls_hi, &r.ls_lo);
    }
    if (pole == 1) {
      r.lc_hi = -std::numeric_limits<double>::infinity();
      r.lc_lo = 0.0;
    } else {
      split(std::log2(ch), &r.lc_hi, &r.lc_lo);
    }
    r.diff = std::sin(th) < (long double)kPoleSin;
    ring[t] = r;
  }

  p->ring0 = 0;
  p->nint = R;
  if (p->sampling == S2GB_MWSS) {             // theta = 0 and pi are rings: exact pole kernels
    p->ring0 = 1; p->nint = L - 1; p->pole_n = 0; p->pole_s = L;
  } else if (p->sampling == S2GB_MW && p->mrec) {   // theta = pi (last ring) likewise
    p->nint = L - 1; p->pole_s = L - 1;
  }
  const int rend = p->ring0 + p->nint;
  p->cap_n = p->ring0;
  while (p->cap_n < rend && ring[p->cap_n].diff) ++p->cap_n;
  p->cap_s = rend;
  while (p->cap_s > p->cap_n && ring[p->cap_s - 1].diff) --p->cap_s;
  p->fwd_parts = (p->nint <= kFwdChunk || p->mrec) ? 1 : 2 + (p->cap_s - p->cap_n + kFwdChunk - 1) / kFwdChunk;

  // ---- starting values d^{l0}_{m,n} (Eq. "initial_values" and Sec. 3.3 symmetries) ----
  std::vector<long double> lf2 = log2_factorials(2 * L + 2);
  std::vector<SeedData> seed((size_t)nN * T);
  for (int ni = 0; ni < nN; ++ni) {
    const int n = n_of[ni];
    const int an = n < 0 ? -n : n;
    for (int mi = 0; mi < T; ++mi) {
      const int m = mi - (L - 1);
      const int am = m < 0 ? -m : m;
      SeedData s{};
      int l0, a, b, sign;
      if (m >= an) {            // d^m_{m,n} = sqrt((2m)!/((m+n)!(m-n)!)) (-sin)^{m-n} cos^{m+n}
        l0 = m; a = m - n; b = m + n; sign = ((m - n) & 1) ? -1 : 1;
      } else if (-m >= an) {    // d^l_{-l,n} = (-1)^{l+n} d^l_{l,-n}
        l0 = -m; a = l0 + n; b = l0 - n; sign = 1;
      } else if (n > am) {      // d^n_{m,n} = (-1)^{m-n} d^n_{n,m}
        l0 = n; a = n - m; b = n + m; sign = 1;
      } else {                  // n < -|m|: d^{|n|}_{m,n} = d^{|n|}_{|n|,-m}
        l0 = -n; a = l0 + m; b = l0 - m; sign = ((l0 + m) & 1) ? -1 : 1;
      }
      long double pl = 0.5L * (lf2[2 * l0] - lf2[a] - lf2[b]);
      split(pl, &s.p_hi, &s.p_lo);
      s.l0 = l0; s.a = a; s.b = b; s.sign = sign;
      seed[(size_t)ni * T + mi] = s;
    }
  }

  // ---- per-degree factors ----
  std::vector<double> sinv((size_t)nN * L), sfwd((size_t)nN * L);
  for (int ni = 0; ni < nN; ++ni)
    for (int l = 0; l < L; ++l) {
      long double c;
      if (p->wigner) {
        sinv[(size_t)ni * L + l] = (double)((2.0L * l + 1.0L) / (8.0L * kPiL * kPiL));
        sfwd[(size_t)ni * L + l] = 1.0;
      } else {
        c = std::sqrt((2.0L * l + 1.0L) / (4.0L * kPiL));
        if (p->spin & 1) c = -c;
        sinv[(size_t)ni * L + l] = (double)c;
        sfwd[(size_t)ni * L + l] = (double)c;
      }
    }

  // ---- ring weights and fine-grid weights of the forward quadrature ----
  // MW / MWSS: fold factors of the torus trapezoid onto the rings (1 on a ring that is its own
  // reflection, theta = 0 or pi; 2 elsewhere).  DH: the DH weights times the phi step.
  std::vector<double> nu(R, 2.0);
  if (p->sampling == S2GB_DH) {
    nu = dh_ring_weights(L);
  } else {
    nu[R - 1] = 1.0;
    if (p->sampling == S2GB_MWSS) nu[0] = 1.0;
  }
  const int NF = p->Nfft;
  const int TS = p->TS;
  std::vector<double> wf(NF);
  if (TS) {
    // W_B(x) = sum_{|k| <= 2L-2} What(k) e^{ikx},  What(0) = 1/pi, What(k) = 1/(pi (1-k^2)) for
    // even k != 0 and 0 for odd k: the Fourier series of |sin x|/2, truncated.  Sampled at
    // x_j = x_0 + 2 pi j/NF with x_0 the first torus point (pi/TS on MW, 0 on MWSS), so that the
    // grid's phase factors cancel; all constants of the pipeline, (2 pi/P)(2 pi/TS)/(TS NF), folded
    // in (see api.cu).
    const int shift = p->sampling == S2GB_MWSS ? 0 : 1;
    const long double cst = (2.0L * kPiL / p->P) * (2.0L * kPiL / TS) / ((long double)TS * NF);
    const long long TN2 = 2LL * TS * NF;
    for (int j = 0; j < NF; ++j) {
      long double acc = 0.0L;
      for (int k = 2; k <= 2 * L - 2; k += 2) {
        // k x_j = pi num / (TS NF)
        long long num = ((long long)k * ((long long)shift * NF + 2LL * j * TS)) % TN2;
        double ang = (double)num * (kPi / ((double)TS * NF));
        acc += (long double)(std::cos(ang) / (1.0 - (double)k * k));
      }
      wf[j] = (double)((1.0L / kPiL + (2.0L / kPiL) * acc) * cst);
    }
  }

  size_t bytes = 0;
  int rc;
  if ((rc = upload(&p->ring, ring, &bytes))) return rc;
  if ((rc = upload(&p->seed, seed, &bytes))) return rc;
  if ((rc = upload(&p->scale_inv, sinv, &bytes))) return rc;
  if ((rc = upload(&p->scale_fwd, sfwd, &bytes))) return rc;
  if ((rc = upload(&p->nu, nu, &bytes))) return rc;
  if ((rc = upload(&p->wfine, wf, &bytes))) return rc;
  if ((rc = upload(&p->n_of, n_of, &bytes))) return rc;
  if (p->mrec) {
    std::vector<double> csc(R, 0.0);
    for (int t = p->ring0; t < p->ring0 + p->nint; ++t) {
      long double th;
      if (p->sampling == S2GB_MWSS) th = (long double)t * kPiL / (long double)L;
      else if (p->sampling == S2GB_DH) th = (long double)(2 * t + 1) * kPiL / (4.0L * L);
      else th = (long double)(2 * t + 1) * kPiL / (long double)T;
      csc[t] = (double)(1.0L / std::sin(th));
    }
    if ((rc = upload(&p->csc, csc, &bytes))) return rc;
    const size_t ab_bytes = (size_t)L * T * 2 * sizeof(double);
    if (cudaMalloc((void**)&p->mrec_ab, ab_bytes) != cudaSuccess) return S2GB_ENOMEM;
    bytes += ab_bytes;
    mrec_ab_kernel<<<1024, 256>>>(p->mrec_ab, L);
    if (launched() != cudaSuccess) return S2GB_ECUDA;
  }
  const int per_step = p->precision == S2GB_FP64 ? kCoefPerStepN : kCoefPerStep;
  const size_t coef_bytes = (size_t)nN * T * L * per_step * sizeof(double);
  if (cudaMalloc((void**)&p->coef, coef_bytes) != cudaSuccess) return S2GB_ENOMEM;
  bytes += coef_bytes;
  p->device_bytes = bytes;
  if (p->precision == S2GB_FP64)
    coefn_kernel<<<(nN * T + 127) / 128, 128>>>(p->coef, p->n_of, nN, L);
  else
    coef_kernel<<<1024, 256>>>(p->coef, p->n_of, nN, L);
  if (launched() != cudaSuccess) return S2GB_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return S2GB_ECUDA;
  if (p->precompute) {
    if ((rc = build_dtable(p, &bytes))) return rc;
    p->device_bytes = bytes;
  }
  if (p->precision == S2GB_FP32) {
    // float32 plans keep the coefficient table rounded once to float, and v per ring
    const size_t n = (size_t)nN * T * L * kCoefPerStep;
    if (cudaMalloc((void**)&p->coef32, n * sizeof(float)) != cudaSuccess) return S2GB_ENOMEM;
    to_float_kernel<<<1024, 256>>>(p->coef, p->coef32, n);
    if (launched() != cudaSuccess) return S2GB_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return S2GB_ECUDA;
    cudaFree(p->coef);
    p->coef = nullptr;
    bytes += n * sizeof(float);
    bytes -= coef_bytes;
    std::vector<float> v32(R);
    for (int t = 0; t < R; ++t) v32[t] = (float)ring[t].v;
    if ((rc = upload(&p->v32, v32, &bytes))) return rc;
    p->device_bytes = bytes;
  }

  // ---- cuFFT plans ----
  const bool f64 = p->precision == S2GB_FP64;
  const cufftType ty = f64 ? CUFFT_Z2Z : CUFFT_C2C;
  const int S[2] = {nN, p->max_batch * nN};
  const int MR = p->MR;
  const int P = p->P;
  for (int q = 0; q < 2; ++q) {
    if (q == 1 && S[1] == S[0]) {
      p->fft_phi[1] = p->fft_phi[0];
      p->fft_phi_c2r[1] = p->fft_phi_c2r[0];
      p->fft_T[1] = p->fft_T[0];
      p->fft_N[1] = p->fft_N[0];
      continue;
    }
    if (p->real) {   // rings of P = 2L-1 real samples <-> orders m = 0 .. L-1
      if ((rc = make_fft(&p->fft_phi[q], P, S[q] * R, 1, P, f64 ? CUFFT_D2Z : CUFFT_R2C, &p->fft_work, L))) return rc;
      if ((rc = make_fft(&p->fft_phi_c2r[q], P, S[q] * R, 1, L, f64 ? CUFFT_Z2D : CUFFT_C2R, &p->fft_work, P))) return rc;
    } else {
      if ((rc = make_fft(&p->fft_phi[q], P, S[q] * R, 1, P, ty, &p->fft_work))) return rc;
    }
    p->fft_made[q] = true;
    if (TS) {
      if ((rc = make_fft(&p->fft_T[q], TS, S[q] * MR, 1, TS, ty, &p->fft_work))) return rc;
      if ((rc = make_fft(&p->fft_N[q], NF, S[q] * MR, 1, NF, ty, &p->fft_work))) return rc;
      p->fft_op_made[q] = true;
    }
  }
  if (p->wigner) {
    const int K = 2 * p->N - 1;
    if ((rc = make_fft(&p->fft_gam[0], K, R * P, R * P, 1, ty, &p->fft_work))) return rc;
    p->fft_gam_made = true;
  }
  return S2GB_OK;
}

void free_plan(Plan* p) {
  cudaFree(p->dtab);
  cudaFree(p->tab_off);
  cudaFree(p->live0);
  cudaFree(p->coef);
  cudaFree(p->coef32);
  cudaFree(p->v32);
  cudaFree(p->ring);
  cudaFree(p->seed);
  cudaFree(p->scale_inv);
  cudaFree(p->scale_fwd);
  cudaFree(p->nu);
  cudaFree(p->wfine);
  cudaFree(p->n_of);
  cudaFree(p->mrec_ab);
  cudaFree(p->csc);
  cudaFree(p->op_dig);
  cudaFree(p->op_rexp);
  cudaFree(p->op_diag);
  for (int q = 0; q < 2; ++q) {
    if (p->fft_made[q]) {
      cufftDestroy(p->fft_phi[q]);
      if (p->real) cufftDestroy(p->fft_phi_c2r[q]);
    }
    if (p->fft_op_made[q]) {
      cufftDestroy(p->fft_T[q]);
      cufftDestroy(p->fft_N[q]);
    }
  }
  if (p->fft_gam_made) cufftDestroy(p->fft_gam[0]);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace regions of a call on `batch` signals (bytes, before alignment):
//   A: phi spectra [S][R][SW] and the fine theta grid [S][MR][Nfft] (forward), ring spectra (inverse)
//   B: theta-torus rows [S][MR][max(T, TS)], or a signal-sized buffer [S][R][SW] (Wigner, DH)
//   C: a second signal-sized buffer (Wigner: the gamma DFT)
//   D: partial coefficients of the ring-chunked forward theta stage (R > kFwdChunk), or the
//      per-CTA partial sums of the order-recursion kernels
// with S = batch * nN and SW = P (complex signals) or L (real signals: orders m >= 0).
void workspace_regions(const Plan& p, int batch, size_t out[4]) {
  const size_t es = p.precision == S2GB_FP64 ? 16 : 8;
  const size_t S = (size_t)batch * p.nN;
  const size_t SW = p.real ? (size_t)p.L : (size_t)p.P;
  const size_t spectra = (size_t)p.R * SW;
  size_t wA = (size_t)p.MR * (size_t)(p.Nfft > p.L ? p.Nfft : p.L);
  if (spectra > wA) wA = spectra;
  size_t wB = (size_t)p.MR * (size_t)(p.TS > p.T ? p.TS : p.T);
  if (spectra > wB) wB = spectra;
  out[0] = S * wA * es;
  out[1] = S * wB * es;
  out[2] = p.wigner ? S * spectra * es : 0;
  out[3] = p.fwd_parts > 1 ? (size_t)p.fwd_parts * S * p.L * (size_t)p.MR * es : 0;
  if (p.mrec) out[3] = mrec_part_bytes(p, batch);
}

size_t workspace_bytes(const Plan& p, int batch) {
  if (batch < 1 || batch > p.max_batch) return 0;
  size_t r[4];
  workspace_regions(p, batch, r);
  return align256(r[0]) + align256(r[1]) + align256(r[2]) + align256(r[3]) + align256(p.fft_work) + 256;
}

}  // namespace s2gb
