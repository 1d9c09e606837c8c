/*
 * s2gb -- spin spherical-harmonic and Wigner transforms on equiangular samplings for NVIDIA
 * GB300 (sm_103a).  C ABI of libs2gb.so.
 *
 * The operations are those of Price & McEwen, "Differentiable and accelerated spherical harmonic
 * and Wigner transforms" (arXiv:2311.14670):
 *   - forward / inverse spin-s spherical-harmonic transform, separated into a phi-DFT and a theta
 *     stage (Sec. 4.1, Eqs. disc_sh_expanded, disc_sh_fft, disc_ish_fft, disc_ish_expanded),
 *     on MW, MWSS and DH sampling (Sec. 4.2);
 *   - forward / inverse Wigner transform as a gamma-DFT plus spin-(-n) transforms (Sec. 2.3, 4.5);
 *   - the adjoints of both directions (Sec. 5.2).
 * The Wigner d-functions of the theta stage are generated on the fly by a three-term recursion
 * in the degree l, interleaved with the theta contraction (Sec. 4.4), and never stored.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *   L      bandlimit (l < L), L >= 1.
 *   T      2L - 1 (number of orders m; number of phi samples on MW and DH).
 *   R, P   rings and phi samples of the plan's sampling (see S2GB_MW below); on MW R = L and
 *          P = T, theta_t = (2t+1) pi / (2L-1), t < L;  phi_p = 2 pi p / (2L-1), p < T.
 *   sY_lm(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi}.
 *   Sphere signal      f  [batch][R][P]              (ring t, sample p), row-major.
 *   Sphere coefficients flm[batch][L][T]             (degree l, index m+L-1).
 *   SO(3) signal       f  [batch][2N-1][R][P]        (gamma_k = 2 pi k/(2N-1), beta_t, alpha_p).
 *   Wigner coefficients flmn[batch][2N-1][L][T]      (index n+N-1, degree l, index m+L-1).
 *   Coefficient entries with |m| > l, or l < |s| (sphere) / l < |n| (Wigner), are ignored on
 *   input and written as 0 on output.
 *   Element type: interleaved complex, double (complex128) for S2GB_FP64 plans and float
 *   (complex64) for S2GB_FP32 plans.  All data pointers are DEVICE pointers on the plan's device,
 *   16-byte aligned (8-byte for complex64).  The caller owns them.
 *   Adjoints are taken with respect to the Euclidean inner product sum conj(x) y (so that
 *   adjoint_inverse(grad_f) is the gradient of a real loss with respect to flm, PyTorch's
 *   convention for complex tensors).
 *
 * Execution model: every transform call only enqueues work on `stream` (a cudaStream_t passed as
 * void*, NULL = legacy default stream) and returns.  It launches kernels and cuFFT executions and
 * allocates nothing.  Scratch memory is the caller's `ws` buffer of at least
 * s2gb_workspace_bytes(plan, batch) bytes; calls that may run concurrently need distinct
 * workspaces.  A plan is immutable after creation; its cuFFT handles are shared, and calls on the
 * same plan from several host threads are serialised internally around the cuFFT executions.
 * Errors are returned as negative codes; no exception crosses the ABI.  Asynchronous kernel
 * faults surface, as in any CUDA program, at the next synchronising call.
 */
#ifndef S2GB_H
#define S2GB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct s2gb_plan_s* s2gb_plan;

/* Return codes. */
enum {
  S2GB_OK = 0,
  S2GB_EINVAL = -1,        /* bad argument: null pointer, size out of range, in == out, ... */
  S2GB_EUNSUPPORTED = -2,  /* valid request that this library does not implement */
  S2GB_ENOMEM = -3,        /* device allocation failed (plan creation only) */
  S2GB_ECUDA = -4,         /* a CUDA runtime call or kernel launch failed */
  S2GB_ECUFFT = -5,        /* a cuFFT call failed */
  S2GB_EWORKSPACE = -6     /* ws is NULL or smaller than s2gb_workspace_bytes() */
};

/*
 * Sampling schemes (Sec. 4.2).  R theta rings by P phi samples, phi_p = 2 pi p / P:
 *   S2GB_MW   McEwen-Wiaux (Sec. 4.2.2): R = L, theta_t = (2t+1) pi/(2L-1), P = 2L-1.
 *   S2GB_MWSS its symmetric variant (Sec. 4.2.2): R = L+1, theta_t = pi t/L (both poles are
 *             rings), P = 2L.
 *   S2GB_DH   Driscoll-Healy (Sec. 4.2.1): R = 2L, theta_t = (2t+1) pi/(4L), P = 2L-1.
 * Every scheme has an exact forward quadrature for bandlimited signals: MW and MWSS through the
 * torus extension of Sec. 4.2.2, DH through its explicit weights.  On MWSS's two pole rings the
 * d-functions are Kronecker deltas (Sec. 3.3); those rings are computed directly and the recursion
 * runs over the L-1 interior rings.
 */
enum { S2GB_MW = 0, S2GB_MWSS = 1, S2GB_DH = 2 };

/* Arithmetic of the theta stage. */
enum {
  S2GB_FP64 = 0,  /* float64 recursion and contraction, complex128 data */
  S2GB_FP32 = 1   /* float32 recursion and contraction with float64 seeds, complex64 data */
};

/*
 * Create a plan on `device` for bandlimit L.
 *   N == 0 : spin-`spin` sphere transforms, |spin| < L.
 *   N >= 1 : Wigner transforms on SO(3) with azimuthal bandlimit N (|n| < N), N <= L; `spin` is
 *            ignored.
 * max_batch >= 1 bounds the `batch` argument of later calls.  The plan holds on the device the
 * recursion coefficient tables (Sec. 3.3 readings, O(L^2) per spin), the per-ring and per-order
 * log-space seed data (Eq. "initial_values") and the FFT weights; it creates cuFFT plans.
 * Returns S2GB_EINVAL for L < 1 or L > 8192, |spin| >= L (sphere), N < 0 or N > L, max_batch < 1,
 * an unknown sampling or precision; S2GB_EUNSUPPORTED for DH with L > 4096, for S2GB_FP32
 * with L > 2048 or DH with L > 1024, and when max_batch * (2N-1 for Wigner plans, else 1) *
 * max(R, 2L-1) exceeds 2^31 - 1 (the FFT stages' 32-bit batch counts);
 * S2GB_ENOMEM / S2GB_ECUDA / S2GB_ECUFFT on device failures.  On failure *out is set to NULL.  The
 * calling thread's current device is restored on return.
 */
int s2gb_plan_create(s2gb_plan* out, int L, int spin, int N, int sampling, int precision,
                     int max_batch, int device);

/*
 * Plan for real signals (spin 0 sphere transforms of real-valued f), whose coefficients obey the
 * Hermitian symmetry flm(l, -m) = (-1)^m conj(flm(l, m)) (Sec. 2.2).  Only the orders m >= 0 are
 * stored and computed:
 *   f   real (double / float) [batch][R][P] (MW and DH sampling; MWSS: S2GB_EUNSUPPORTED),
 *   flm complex [batch][L][L], flm[b][l][m] for 0 <= m < L (entries m > l ignored / written 0);
 *       the imaginary parts of flm[b][l][0] are ignored (they are 0 for a real signal).
 * s2gb_forward / s2gb_inverse / the adjoints / the order-range calls take these layouts; the
 * adjoints are with respect to the real inner product Re sum conj(x) y (PyTorch's convention for
 * gradients of real losses).  The theta stages alone use ring spectra [batch][R][L] (column m) and
 * forward-theta input g [batch][L (m)][R (t)].  The theta recursion runs for m >= 0 only and the
 * phi DFTs are real-to-complex / complex-to-real, so a real transform costs about half a complex
 * one.  Arguments as in s2gb_plan_create (spin 0, N = 0 implied).  s2gb_inverse_noalloc refuses
 * real plans (S2GB_EUNSUPPORTED).
 */
int s2gb_plan_create_real(s2gb_plan* out, int L, int sampling, int precision, int max_batch, int device);

/*
 * Plan with options (bitwise OR of the flags below; other bits: S2GB_EINVAL).  flags = 0 is
 * s2gb_plan_create; S2GB_PLAN_REAL is s2gb_plan_create_real (spin and N must be 0).
 *
 * S2GB_PLAN_PRECOMPUTE: precompute mode (Sec. 4.4's precompute variant).  At plan creation the
 * Wigner d-functions d^l_{m,n}(theta_t) on the L MW rings are generated by the plan's recursion
 * and kept in device memory; every transform (and adjoint, order-range and theta-only call) then
 * reads them instead of recomputing them.  Same results to rounding (|d| < 2^-400 is stored as 0,
 * as the on-the-fly kernels skip such values).  Memory: 8 bytes x L rings x the (l, m, n) triples
 * the theta kernels run -- with the +-m pairing of spin-0 and Wigner plans only m >= 0 at n = 0
 * (L = 1024 spin 0: 4.3 GB; spin 2: 8.6 GB; L = 2048 spin 0: 34 GB; real plans as spin 0);
 * s2gb_plan_device_bytes includes it.  FP64 MW plans with L <= 2048 only (else S2GB_EUNSUPPORTED);
 * S2GB_ENOMEM when the table does not fit.
 *
 * S2GB_PLAN_MRECURSION: the theta stages generate the d-functions with the paper's own recursion
 * over the order m (Sec. 3.3, Eq. wigner-d-recursion: downward from m = l, started from Eq.
 * initial_values, run independently for every (l, theta)) instead of the default recursion over
 * the degree l.  Same results to rounding; every transform and adjoint of sphere and Wigner plans
 * (FP64 only; not with S2GB_PLAN_REAL or S2GB_PLAN_PRECOMPUTE: S2GB_EUNSUPPORTED).  Each (l, theta)
 * runs two chains -- at theta for m >= rint(n cos theta) and at pi - theta for the rest, through
 * d^l_{m,n}(theta) = (-1)^{l+n} d^l_{-m,n}(pi - theta) -- so that no chain crosses its lower
 * turning point; the ring theta = pi (and theta = 0), where the recursion coefficient is
 * undefined, takes the closed forms of Sec. 3.3.  Because m is both the recursion index and the
 * output index of the contraction, the kernels sum across threads and write per-block partial
 * sums into the workspace (s2gb_workspace_bytes includes them); the theta-only entry points and
 * s2gb_inverse_noalloc return S2GB_EUNSUPPORTED for these plans.
 *
 * S2GB_PLAN_FMA_CONTRACTION: float64 plans whose d-functions are generated on the fly (neither
 * PRECOMPUTE nor MRECURSION) run the theta contraction -- the sum over the degree l of the inverse
 * stage (Eq. disc_ish_expanded) and over the rings of the forward (Eq. disc_sh_expanded) -- on the
 * tensor cores by default: the float64 recursion values and the coefficients are split into seven
 * exact base-256 digits each, whose products the tensor cores sum exactly in float32 (the Ozaki
 * splitting scheme); the digit sums are combined in 64-bit integers and float64.  The result
 * agrees with a float64 sum to a few units of the last place.  Float32 plans with max_batch >= 16
 * run their inverse theta stage the same way with four digits (a float32 value to 2^-30 of its
 * bound) and exact integer level sums in place of compensated float32 sums, for every call on the
 * plan (smaller float32 plans keep the FMA pipe, which is faster for few signals).  This flag keeps
 * the contraction on the FMA pipe instead (float64 or float32; for comparison).  Ignored by other
 * plans.
 */
#define S2GB_PLAN_REAL 1u
#define S2GB_PLAN_PRECOMPUTE 2u
#define S2GB_PLAN_MRECURSION 4u
#define S2GB_PLAN_FMA_CONTRACTION 8u
int s2gb_plan_create_flags(s2gb_plan* out, int L, int spin, int N, int sampling, int precision,
                           int max_batch, int device, unsigned flags);

/* Free a plan and everything it holds (NULL is ignored).  No call on it may be in flight. */
void s2gb_plan_destroy(s2gb_plan plan);

/* Bytes of scratch a transform call on `batch` signals needs (0 if batch is out of range). */
size_t s2gb_workspace_bytes(s2gb_plan plan, int batch);

/* Bytes of device memory the plan itself holds (tables, weights, cuFFT plans excluded). */
size_t s2gb_plan_device_bytes(s2gb_plan plan);

/*
 * Forward transform (Sec. 4.1, Eqs. disc_sh_fft + disc_sh_expanded; Wigner: Eq. wigner_sht_forward
 * with the gamma-DFT).  f -> flm.  The theta quadrature is exact for bandlimited signals (the
 * sampling theorems of Sec. 4.2).  f and flm must not overlap (else S2GB_EINVAL).
 */
int s2gb_forward(s2gb_plan plan, const void* f, void* flm, int batch, void* ws, size_t ws_bytes,
                 void* stream);

/* Inverse transform (Eqs. disc_ish_expanded + disc_ish_fft; Wigner: Eq. wigner_sht_inverse). */
int s2gb_inverse(s2gb_plan plan, const void* flm, void* f, int batch, void* ws, size_t ws_bytes,
                 void* stream);

/* Adjoint of s2gb_forward: flm_bar -> f_bar (Sec. 5.2.1, F^H; exact transpose of the pipeline). */
int s2gb_adjoint_forward(s2gb_plan plan, const void* flm_bar, void* f_bar, int batch, void* ws,
                         size_t ws_bytes, void* stream);

/* Adjoint of s2gb_inverse: f_bar -> flm_bar (Sec. 5.2.2, F^{-H}). */
int s2gb_adjoint_inverse(s2gb_plan plan, const void* f_bar, void* flm_bar, int batch, void* ws,
                         size_t ws_bytes, void* stream);

/*
 * Theta stages alone (the recursion + contraction kernels, Sec. 4.4), for sphere plans.
 *
 * s2gb_inverse_theta: Eq. disc_ish_expanded,
 *     ftilde[b][t][k] = sum_l (-1)^s sqrt((2l+1)/(4 pi)) flm[b][l][m+L-1] d^l_{m,-s}(theta_t),
 *   ftilde of shape [batch][R][P], k = m mod P (the layout a length-P inverse DFT along the last
 *   axis turns into f); on MWSS the column k = L (no order) is written 0.
 * s2gb_forward_theta: Eq. disc_sh_expanded on the R rings of the sampling with ring weights
 *   already applied,
 *     flm[b][l][m+L-1] = (-1)^s sqrt((2l+1)/(4 pi)) sum_t d^l_{m,-s}(theta_t) g[b][m+L-1][t],
 *   g of shape [batch][T][R] (order-major).
 * Same pointer, batch and stream rules as the transforms; no workspace is needed.  For N >= 1
 * plans these return S2GB_EUNSUPPORTED, and so does s2gb_forward_theta when the recursion runs over
 * more than 2048 rings (its ring chunks need the transforms' workspace).
 */
int s2gb_inverse_theta(s2gb_plan plan, const void* flm, void* ftilde, int batch, void* stream);
int s2gb_forward_theta(s2gb_plan plan, const void* g, void* flm, int batch, void* stream);

/*
 * Order-sharded transforms: one transform split over devices (or over sequential calls) by |m|.
 * For a fixed order m, flm[.][m] <-> ftilde_m(theta) is a closed subproblem in both directions
 * (Eqs. disc_ish_expanded and disc_sh_expanded couple degrees and rings, never orders), so a
 * device that owns the orders with |m| in [m_lo, m_hi) (0 <= m_lo <= m_hi <= L, else S2GB_EINVAL;
 * m_lo == m_hi is an empty range and launches nothing) computes exactly the values the whole
 * transform computes for those orders, bit for bit.
 *
 * s2gb_inverse_theta_mrange: s2gb_inverse_theta for the orders in range only (sphere plans).
 *   Columns of ftilde for other orders are not written (on MWSS the column k = L is written 0).
 * s2gb_inverse_phi: the rest of the sphere inverse transform, ftilde [b][t][m mod P] -> f
 *   (Eq. disc_ish_fft, a length-P inverse DFT along phi).  Sphere plans (Wigner:
 *   S2GB_EUNSUPPORTED); workspace as for s2gb_inverse.  s2gb_inverse = s2gb_inverse_theta +
 *   s2gb_inverse_phi; an order-sharded inverse assembles ftilde from every shard (one exchange of
 *   16 * batch * R * P bytes in FP64) before s2gb_inverse_phi.
 * s2gb_forward_mrange: s2gb_forward whose theta stage runs for the orders in range only; every
 *   stage before it (the phi DFT and the theta-direction quadrature operator) runs in full.
 *   flm entries of other orders are not written.  Any plan (sphere or Wigner); workspace as for
 *   s2gb_forward.
 * Same pointer, batch and stream rules as the transforms.
 */
int s2gb_inverse_theta_mrange(s2gb_plan plan, const void* flm, void* ftilde, int batch, int m_lo,
                              int m_hi, void* stream);
int s2gb_inverse_phi(s2gb_plan plan, const void* ftilde, void* f, int batch, void* ws, size_t ws_bytes,
                     void* stream);
int s2gb_forward_mrange(s2gb_plan plan, const void* f, void* flm, int batch, int m_lo, int m_hi,
                        void* ws, size_t ws_bytes, void* stream);

/*
 * Allocation-free inverse transform.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory at the point where they run the transform -- code
 * whose memory is owned by another allocator, code running under a strict no-allocation rule
 * (real-time or certified pipelines), or plugins that are handed only their input and output.
 * It computes exactly what s2gb_inverse computes (same arguments, layouts and results) but takes
 * no workspace: its scratch is a static device array of S2GB_NOALLOC_SCRATCH_BYTES inside
 * libs2gb.so, which every GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc / cudaFree and no allocating library routine (the plan must already exist).
 *   - Returns S2GB_EWORKSPACE when the call needs more scratch than the array holds: the
 *     theta-stage output (batch * R * P elements; three such buffers for Wigner plans) plus
 *     the cuFFT work area of the phi (and gamma) DFT.  With complex128 data, 64 MiB covers for
 *     example L = 1024 with batch 1 or L = 512 with batch 4.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any CUDA stream capture.
 *   - Every call shares the one array and it keeps the previous call's contents (this transform
 *     overwrites everything it reads back, so nothing needs clearing).  Calls that may overlap on
 *     the GPU (different streams, different host threads without ordering) race on it: serialise
 *     them.
 */
#define S2GB_NOALLOC_SCRATCH_BYTES (64u << 20)
int s2gb_inverse_noalloc(s2gb_plan plan, const void* flm, void* f, int batch, void* stream);

/*
 * Number of kernel launches of this library (its own kernels; cuFFT's are not counted) issued by
 * the calling process since the library was loaded, plan-creation kernels included.  A host-side
 * counter, incremented when a launch is enqueued; thread-safe; never fails.  Instrumentation only:
 * the paper has no counterpart.
 */
unsigned long long s2gb_kernels_launched(void);

/*
 * Measurement helper (the paper has no counterpart): enqueues one launch of `blocks` x `threads`
 * threads (threads a multiple of 32, at most 256) in which every thread runs
 * s2gb_fma_chain_lanes() independent fused multiply-add chains of `iters` steps in float64
 * (precision S2GB_FP64) or float32 (S2GB_FP32), and writes one value per thread to `out` (device,
 * blocks * threads elements of that type).  The launch performs
 * blocks * threads * s2gb_fma_chain_lanes() * iters FMAs; timed with CUDA events it measures the
 * FMA pipe's throughput, the denominator of the theta kernels' roofline fraction.  Returns
 * S2GB_EINVAL on bad sizes.
 */
int s2gb_fma_chain(int precision, int blocks, int threads, long long iters, void* out, void* stream);
int s2gb_fma_chain_lanes(void);

/*
 * Status of the tensor-core theta kernels on `device` (the paper has no counterpart): 0 when every
 * such kernel finished normally; otherwise the code recorded by the first kernel whose bounded wait
 * for tensor-core completion ran out (1) -- that kernel left its output unwritten.  Synchronous
 * (reads a device variable); `clear` != 0 resets the status to 0.  Negative return: S2GB_EINVAL
 * (no such device) or S2GB_ECUDA.
 */
int s2gb_device_status(int device, int clear);

/* Static description of a return code (never NULL). */
const char* s2gb_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* S2GB_H */
