"""Spin-s spherical-harmonic and Wigner transforms on MW sampling -- the oracle (test infrastructure).

Everything is a direct sum in float64 (no FFT); exponentials are built from exactly reduced
integer phases.  ``exact=True`` (sphere transforms on every sampling, MW Wigner transforms)
runs the same algorithm with the d-functions, weights, phases and every sum in numpy's extended
precision (np.longdouble: 80-bit on x86-64, binary128 on aarch64) and rounds once to complex128 at
the end (``keep=True`` returns the extended-precision result).  Array conventions (shared with the GPU library's boundary, written out here
independently):

* sphere signal   f[..., t, p]           t < L rings (theta_t), p < 2L-1 (phi_p)
* coefficients    flm[..., l, m+L-1]     l < L, |m| <= l; other entries ignored / returned as 0
* SO(3) signal    f[..., k, t, p]        k < 2N-1 (gamma_k = 2 pi k/(2N-1)), t (beta), p (alpha)
* Wigner coeffs   flmn[..., n+N-1, l, m+L-1]

Definitions followed (Sec. 4.1): with c_l = (-1)^s sqrt((2l+1)/(4 pi)),
  inverse  (Eqs. disc_ish_expanded, disc_ish_fft):
      f~_m(theta) = sum_l c_l flm_lm d^l_{m,-s}(theta),   f(theta, phi_p) = sum_m f~_m(theta) e^{i m phi_p}
  forward  (Eqs. disc_sh_fft, disc_sh_expanded; Sec. 4.2.2 for MW):
      F_m(theta_t) = sum_p f(theta_t, phi_p) e^{-i m phi_p}
      extend to the theta torus: G_m(theta_{2L-2-t}) = (-1)^{m+s} F_m(theta_t), and at the
      self-reflected ring theta = pi, G_m(pi) = (1 + (-1)^{m+s})/2 F_m(pi) (reading, see _extend)
      upsample to the MW grid of bandlimit 2L by zero padding the theta-Fourier series
      flm_lm = c_l sum_u q_u d^l_{m,-s}(theta'_u) q_Phi G_m(theta'_u),   q_Phi = 2 pi/(2L-1)
The Wigner transform (Sec. 2.3, 4.5) is a gamma-DFT plus spin-(-n) transforms whose per-l factor
is (2l+1)/(8 pi^2) (inverse) or 1 (forward) instead of c_l.  Adjoints (Sec. 5.2) are the
conjugate transposes of these linear maps, written stage by stage in reverse order.
"""
from __future__ import annotations

import numpy as np

from .sampling import (dh_theta_weights, dh_thetas, mw_theta_weights, mw_thetas, mwss_theta_weights,
                       mwss_thetas)
from .wigner import PI_LD, wigner_d_table

_CHUNK_BYTES = 256 << 20


def _cdtype(dtype):
    """The complex type of a real type (float64 -> complex128, longdouble -> clongdouble)."""
    return np.clongdouble if dtype == np.longdouble else np.complex128


def _expi_pi(num, den: int, dtype=np.float64) -> np.ndarray:
    """exp(i pi num/den) for integer arrays num, reduced exactly modulo 2 den."""
    r = np.mod(np.asarray(num, dtype=np.int64), 2 * den)
    ang = r.astype(np.longdouble) * PI_LD / np.longdouble(den)
    out = np.empty(ang.shape, dtype=np.clongdouble)
    out.real = np.cos(ang)
    out.imag = np.sin(ang)
    return out.astype(_cdtype(dtype))


def phi_dft_matrix(L: int, sign: int, dtype=np.float64) -> np.ndarray:
    """E[p, j] = exp(sign * i m_j phi_p), m_j = j - (L-1), phi_p = 2 pi p/(2L-1)."""
    T = 2 * L - 1
    p = np.arange(T)[:, None]
    m = np.arange(-(L - 1), L)[None, :]
    return _expi_pi(sign * 2 * p * m, T, dtype)


def ell_factor(L: int, spin: int, dtype=np.float64) -> np.ndarray:
    """c_l = (-1)^s sqrt((2l+1)/(4 pi)), l < L (Eq. disc_sh_expanded)."""
    ell = np.arange(L).astype(np.longdouble)
    return ((-1.0) ** spin * np.sqrt((2 * ell + 1) / (4 * PI_LD))).astype(dtype)


def coeff_mask(L: int, n: int) -> np.ndarray:
    """True where max(|m|, |n|) <= l < L, shape (L, 2L-1)."""
    ell = np.arange(L)[:, None]
    m = np.arange(-(L - 1), L)[None, :]
    return (np.abs(m) <= ell) & (abs(n) <= ell)


# ----------------------------------------------------------------------------- inverse
def _theta_inverse(flm: np.ndarray, L: int, n: int, scale: np.ndarray, thetas, dtype=np.float64) -> np.ndarray:
    """f~[..., t, m] = sum_l scale_l flm[..., l, m] d^l_{m,n}(theta_t) (Eq. disc_ish_expanded)."""
    flm = np.where(coeff_mask(L, n), flm, 0) * scale[:, None]
    out = np.zeros(flm.shape[:-2] + (len(thetas), 2 * L - 1), dtype=_cdtype(dtype))
    per_ring = L * (2 * L - 1) * np.dtype(dtype).itemsize
    step = max(1, _CHUNK_BYTES // per_ring)
    for a in range(0, len(thetas), step):
        D = wigner_d_table(np.arange(L), n, thetas[a:a + step], dtype)   # [l, m, t]
        out[..., a:a + step, :] = np.einsum("...lm,lmt->...tm", flm, D)
    return out


def _finish(x: np.ndarray, keep: bool) -> np.ndarray:
    """The result as complex128, or as computed when ``keep``."""
    return x if keep else x.astype(np.complex128)


def inverse(flm: np.ndarray, L: int, spin: int, rings=None, exact: bool = False, keep: bool = False) -> np.ndarray:
    """Inverse spin-s SHT on the MW grid; ``rings`` selects theta indices (default: all L).
    ``exact``: extended-precision d-functions and sums (module docstring)."""
    dt = np.longdouble if exact else np.float64
    th = mw_thetas(L)
    if rings is not None:
        th = th[np.asarray(rings)]
    ft = _theta_inverse(np.asarray(flm).astype(_cdtype(dt)), L, -spin, ell_factor(L, spin, dt), th, dt)
    return _finish(ft @ phi_dft_matrix(L, +1, dt).T, keep)               # Eq. disc_ish_fft


# ----------------------------------------------------------------------------- forward
def _upsample_matrices(L: int, dtype=np.float64):
    """Matrices of the theta torus extension / Fourier coefficients / upsampled evaluation."""
    T = 2 * L - 1
    Tu = 4 * L - 1                       # torus length of the MW grid at bandlimit 2L
    k = np.arange(-(L - 1), L)
    tt = np.arange(T)
    uu = np.arange(2 * L)
    coef = _expi_pi(-np.outer(k, 2 * tt + 1), T, dtype) / dtype(T)        # [k, t'] e^{-ik theta_t'}/T
    up = _expi_pi(np.outer(2 * uu + 1, k), Tu, dtype)                       # [u, k]  e^{+ik theta'_u}
    return coef, up


def _phi_forward(f: np.ndarray, L: int, orders=None, dtype=np.float64) -> np.ndarray:
    """F[..., t, m] = sum_p f[..., t, p] e^{-i m phi_p} (Eq. disc_sh_fft without q_Phi).

    ``orders``: optional subset of the orders m (default: all |m| < L, in increasing order)."""
    E = phi_dft_matrix(L, -1, dtype)
    if orders is not None:
        E = E[:, np.asarray(orders) + L - 1]
    return np.asarray(f).astype(_cdtype(dtype)) @ E


def _extend(F: np.ndarray, L: int, n: int, orders=None) -> np.ndarray:
    """Torus extension in theta, G[..., t', m] for t' < 2L-1 (Sec. 4.2.2); n is the d-index (-s).

    Reading: the ring theta = pi is its own reflection, so the extension there is the average of
    the ring and its reflection, G_m(pi) = (1 + (-1)^{m+s})/2 F_m(pi).  Bandlimited signals already
    have F_m(pi) = 0 for odd m+s; for arbitrary samples this makes the torus function exactly of
    parity (-1)^{m+s}, so that every exact theta quadrature gives the same result."""
    m = np.arange(-(L - 1), L) if orders is None else np.asarray(orders)
    sigma = (-1.0) ** ((m - n) % 2)                                         # (-1)^{m+s}
    G = np.zeros(F.shape[:-2] + (2 * L - 1, F.shape[-1]), dtype=F.dtype)
    G[..., :L, :] = F
    G[..., L - 1, :] = F[..., L - 1, :] * (1 + sigma) / 2
    G[..., L:, :] = (F[..., :L - 1, :] * sigma)[..., ::-1, :]               # G[2L-2-t] = sigma F[t]
    return G


def _theta_forward_upsampled(Gu: np.ndarray, L: int, n: int, scale: np.ndarray, ells,
                             orders=None, dtype=np.float64) -> np.ndarray:
    """flm[..., i, m] = scale_l sum_u q_u d^l_{m,n}(theta'_u) q_Phi Gu[..., u, m], l = ells[i]."""
    ells = np.asarray(ells)
    mcols = np.arange(2 * L - 1) if orders is None else np.asarray(orders) + L - 1
    q = mw_theta_weights(2 * L, dtype)
    qphi = (2 * PI_LD / (2 * L - 1)).astype(dtype)
    thu = mw_thetas(2 * L)
    W = Gu * (q * qphi)[:, None]
    out = np.zeros(Gu.shape[:-2] + (len(ells), len(mcols)), dtype=_cdtype(dtype))
    per_l = (2 * L - 1) * 2 * L * np.dtype(dtype).itemsize * 2
    step = max(1, _CHUNK_BYTES // per_l)
    for a in range(0, len(ells), step):
        sel = ells[a:a + step]
        D = wigner_d_table(sel, n, thu, dtype)                               # [i, m', u], m' width max(sel)
        M = int(sel.max())
        D = D[:, M - (L - 1):M + L, :] if M >= L - 1 else np.pad(D, ((0, 0), (L - 1 - M, L - 1 - M), (0, 0)))
        out[..., a:a + step, :] = np.einsum("...um,imu->...im", W, D[:, mcols, :]) * scale[sel][:, None]
    mask = coeff_mask(L, n)[ells][:, mcols]
    return np.where(mask, out, 0)


def forward(f: np.ndarray, L: int, spin: int, ells=None, orders=None, exact: bool = False,
            keep: bool = False) -> np.ndarray:
    """Forward spin-s SHT on the MW grid; ``ells`` selects output rows (default: all l < L) and
    ``orders`` output columns by order m (default: all |m| < L).  ``exact``: extended-precision
    d-functions, weights and sums (module docstring)."""
    dt = np.longdouble if exact else np.float64
    if ells is None:
        ells = np.arange(L)
    coef, up = _upsample_matrices(L, dt)
    G = _extend(_phi_forward(f, L, orders, dt), L, -spin, orders)
    Gu = up @ (coef @ G)
    return _finish(_theta_forward_upsampled(Gu, L, -spin, ell_factor(L, spin, dt), ells, orders, dt), keep)


# ----------------------------------------------------------------------------- adjoints (Sec. 5.2)
def adjoint_inverse(fbar: np.ndarray, L: int, spin: int) -> np.ndarray:
    """Conjugate transpose of ``inverse``: flm_bar[l, m] = c_l sum_t d^l_{m,-s}(theta_t) sum_p fbar e^{-i m phi_p}."""
    v = _phi_forward(fbar, L)                                                # phi-DFT^H of the synthesis
    th = mw_thetas(L)
    n = -spin
    out = np.zeros(v.shape[:-2] + (L, 2 * L - 1), dtype=np.complex128)
    D = wigner_d_table(np.arange(L), n, th)                                  # [l, m, t]
    out = np.einsum("...tm,lmt->...lm", v, D) * ell_factor(L, spin)[:, None]
    return np.where(coeff_mask(L, n), out, 0)


def adjoint_forward(flm_bar: np.ndarray, L: int, spin: int) -> np.ndarray:
    """Conjugate transpose of ``forward``: every stage of ``forward`` transposed, in reverse order."""
    n = -spin
    flm_bar = np.where(coeff_mask(L, n), np.asarray(flm_bar, dtype=np.complex128), 0)
    q = mw_theta_weights(2 * L)
    qphi = 2 * np.pi / (2 * L - 1)
    thu = mw_thetas(2 * L)
    D = wigner_d_table(np.arange(L), n, thu)                                 # [l, m, u]
    X = np.einsum("...lm,lmu->...um", flm_bar * ell_factor(L, spin)[:, None], D)
    X = X * (q * qphi)[:, None]
    coef, up = _upsample_matrices(L)
    Gbar = coef.conj().T @ (up.conj().T @ X)                                 # [t', m]
    m = np.arange(-(L - 1), L)
    sigma = (-1.0) ** ((m - n) % 2)
    Fbar = Gbar[..., :L, :].copy()
    Fbar[..., L - 1, :] *= (1 + sigma) / 2
    Fbar[..., :L - 1, :] += sigma * Gbar[..., L:, :][..., ::-1, :]
    return Fbar @ phi_dft_matrix(L, -1).conj().T                            # phi-DFT^H


# ----------------------------------------------------------------------------- MWSS and DH (Sec. 4.2)
# Signals on the MWSS grid are f[..., t, p] with t = 0..L (L+1 rings, both poles) and p < 2L; on the
# DH grid t < 2L and p < 2L-1.  Coefficients as for MW.
SAMPLINGS = ("mw", "mwss", "dh")


def sampling_shape(L: int, sampling: str) -> tuple:
    """(rings, phi samples) of a sampling scheme."""
    return {"mw": (L, 2 * L - 1), "mwss": (L + 1, 2 * L), "dh": (2 * L, 2 * L - 1)}[sampling]


def sampling_thetas(L: int, sampling: str):
    return {"mw": mw_thetas, "mwss": mwss_thetas, "dh": dh_thetas}[sampling](L)


def _phi_matrix(L: int, Tp: int, sign: int, dtype=np.float64) -> np.ndarray:
    """E[p, j] = exp(sign i m_j phi_p), m_j = j - (L-1), phi_p = 2 pi p / Tp."""
    p = np.arange(Tp)[:, None]
    m = np.arange(-(L - 1), L)[None, :]
    return _expi_pi(sign * 2 * p * m, Tp, dtype)


def inverse_s(flm: np.ndarray, L: int, spin: int, sampling: str = "mw", rings=None, exact: bool = False,
              keep: bool = False) -> np.ndarray:
    """Inverse spin-s SHT on any of the samplings: the direct sums of Eqs. disc_ish_expanded and
    disc_ish_fft at that grid's theta_t and phi_p.  ``exact``: extended precision (module
    docstring)."""
    if sampling == "mw":
        return inverse(flm, L, spin, rings, exact, keep)
    dt = np.longdouble if exact else np.float64
    th = sampling_thetas(L, sampling)
    if rings is not None:
        th = th[np.asarray(rings)]
    ft = _theta_inverse(np.asarray(flm).astype(_cdtype(dt)), L, -spin, ell_factor(L, spin, dt), th, dt)
    return _finish(ft @ _phi_matrix(L, sampling_shape(L, sampling)[1], +1, dt).T, keep)


def _mwss_extend(F: np.ndarray, L: int, n: int) -> np.ndarray:
    """MWSS torus extension G[..., t', m], t' < 2L: G[t'] = F[t'] (t' <= L), G[2L-t] = sigma F[t]
    (0 < t < L), and at the two self-reflected rings (the poles) the average (1 + sigma)/2 F, as for
    MW's theta = pi ring (same reading)."""
    m = np.arange(-(L - 1), L)
    sigma = (-1.0) ** ((m - n) % 2)
    G = np.zeros(F.shape[:-2] + (2 * L, F.shape[-1]), dtype=F.dtype)
    G[..., :L + 1, :] = F
    G[..., 0, :] = F[..., 0, :] * (1 + sigma) / 2
    G[..., L, :] = F[..., L, :] * (1 + sigma) / 2
    G[..., L + 1:, :] = (F[..., 1:L, :] * sigma)[..., ::-1, :]
    return G


def _sampled_weighted_spectra(f: np.ndarray, L: int, n: int, sampling: str, dtype=np.float64):
    """W[..., u, m] and theta_u such that flm = scale_l sum_u W[u, m] d^l_{m,n}(theta_u) on the MWSS
    or DH grid (f[..., t, p]): the phi DFT, then the theta quadrature of the sampling.
    DH: the explicit DH weights (Sec. 4.2.1).  MWSS: the route of Sec. 4.2.2 -- torus extension,
    Fourier coefficients |k| <= L-1 on the 2L torus points, evaluation on the MWSS grid of
    bandlimit 2L, MWSS weights at bandlimit 2L."""
    Tp = sampling_shape(L, sampling)[1]
    F = np.asarray(f).astype(_cdtype(dtype)) @ _phi_matrix(L, Tp, -1, dtype)  # [t, m]
    qphi = (2 * PI_LD / Tp).astype(dtype)
    if sampling == "dh":
        return F * (dh_theta_weights(L, dtype) * qphi)[:, None], dh_thetas(L)
    G = _mwss_extend(F, L, n)                                                # [t', m], t' < 2L
    k = np.arange(-(L - 1), L)
    coef = _expi_pi(-np.outer(k, 2 * np.arange(2 * L)), 2 * L, dtype) / dtype(2 * L)   # e^{-ik pi t'/L}/2L
    u = np.arange(2 * L + 1)
    up = _expi_pi(np.outer(u, k), 2 * L, dtype)                              # e^{+ik pi u/(2L)}
    Gu = up @ (coef @ G)
    return Gu * (mwss_theta_weights(2 * L, dtype) * qphi)[:, None], mwss_thetas(2 * L)


def _quadrature(W: np.ndarray, thetas, L: int, n: int, scale: np.ndarray, ells, dtype=np.float64) -> np.ndarray:
    """flm[..., i, m] = scale_l sum_u W[..., u, m] d^l_{m,n}(theta_u), l = ells[i] (Eq. disc_sh_expanded)."""
    ells = np.asarray(ells)
    D = wigner_d_table(ells, n, thetas, dtype)                               # [i, m', u]
    M = int(ells.max())
    D = D[:, M - (L - 1):M + L, :] if M >= L - 1 else np.pad(D, ((0, 0), (L - 1 - M, L - 1 - M), (0, 0)))
    out = np.einsum("...um,imu->...im", W, D) * scale[ells][:, None]
    return np.where(coeff_mask(L, n)[ells], out, 0)


def _forward_sampled(f: np.ndarray, L: int, n: int, scale: np.ndarray, sampling: str, ells,
                     dtype=np.float64) -> np.ndarray:
    """flm[..., i, m] = scale_l int f(theta, phi) d^l_{m,n}(theta) e^{-i m phi} sin(theta), l = ells[i],
    on the MWSS or DH grid."""
    W, th = _sampled_weighted_spectra(f, L, n, sampling, dtype)
    return _quadrature(W, th, L, n, scale, ells, dtype)


def forward_s(f: np.ndarray, L: int, spin: int, sampling: str = "mw", ells=None, exact: bool = False,
              keep: bool = False) -> np.ndarray:
    """Forward spin-s SHT on any of the samplings (MW: ``forward``; MWSS, DH: _forward_sampled
    with d^l_{m,-s} and c_l).  ``exact``: extended precision (module docstring)."""
    if sampling == "mw":
        return forward(f, L, spin, ells, None, exact, keep)
    dt = np.longdouble if exact else np.float64
    if ells is None:
        ells = np.arange(L)
    return _finish(_forward_sampled(f, L, -spin, ell_factor(L, spin, dt), sampling, ells, dt), keep)


def adjoint_dense(fn, x_shape, y: np.ndarray) -> np.ndarray:
    """A^H y for the linear map x -> fn(x) (complex-linear), by building A column by column from
    unit vectors: the definition of the adjoint, for small sizes."""
    size = int(np.prod(x_shape))
    cols = [np.asarray(fn(np.eye(1, size, i, dtype=np.complex128).reshape(x_shape))).ravel()
            for i in range(size)]
    A = np.stack(cols, axis=1)
    return (A.conj().T @ np.asarray(y).ravel()).reshape(x_shape)


# ----------------------------------------------------------------------------- real signals (Sec. 2.2)
# A real spin-0 signal has Hermitian coefficients flm_{l,-m} = (-1)^m conj(flm_{lm}) (Sec. 2.2), so
# the orders m >= 0 carry everything: flm_pos[..., l, m] for 0 <= m < L.  The real transforms are
# the complex ones restricted to such signals; as maps between real vector spaces their adjoints
# are taken with respect to the real inner product Re sum conj(x) y.
def hermitian_expand(flm_pos: np.ndarray, L: int) -> np.ndarray:
    """Full coefficients [..., l, m+L-1] from the orders m >= 0 (the real part of m = 0 is used)."""
    flm_pos = np.asarray(flm_pos, dtype=np.complex128)
    out = np.zeros(flm_pos.shape[:-1] + (2 * L - 1,), dtype=np.complex128)
    m = np.arange(1, L)
    out[..., L - 1] = flm_pos[..., 0].real
    out[..., L - 1 + m] = flm_pos[..., m]
    out[..., L - 1 - m] = ((-1.0) ** m) * np.conj(flm_pos[..., m])
    return np.where(coeff_mask(L, 0), out, 0)


def inverse_real(flm_pos: np.ndarray, L: int, sampling: str = "mw") -> np.ndarray:
    """Real signal f[..., t, p] with coefficients hermitian_expand(flm_pos)."""
    return inverse_s(hermitian_expand(flm_pos, L), L, 0, sampling).real


def forward_real(f: np.ndarray, L: int, sampling: str = "mw") -> np.ndarray:
    """Orders m >= 0 of the coefficients of a real signal: flm_pos[..., l, m]."""
    return forward_s(np.asarray(f, dtype=np.float64).astype(np.complex128), L, 0, sampling)[..., L - 1:]


def adjoint_inverse_real(fbar: np.ndarray, L: int) -> np.ndarray:
    """Adjoint of inverse_real: the adjoint of hermitian_expand applied to adjoint_inverse."""
    w = adjoint_inverse(np.asarray(fbar, dtype=np.float64).astype(np.complex128), L, 0)
    m = np.arange(1, L)
    out = np.zeros(w.shape[:-1] + (L,), dtype=np.complex128)
    out[..., 0] = w[..., L - 1].real
    out[..., m] = w[..., L - 1 + m] + ((-1.0) ** m) * np.conj(w[..., L - 1 - m])
    return np.where(coeff_mask(L, 0)[:, L - 1:], out, 0)


def adjoint_forward_real(flm_bar_pos: np.ndarray, L: int) -> np.ndarray:
    """Adjoint of forward_real: the real part of adjoint_forward of the zero-padded orders."""
    flm_bar_pos = np.asarray(flm_bar_pos, dtype=np.complex128)
    full = np.zeros(flm_bar_pos.shape[:-1] + (2 * L - 1,), dtype=np.complex128)
    full[..., L - 1:] = flm_bar_pos
    return adjoint_forward(full, L, 0).real


# ----------------------------------------------------------------------------- Wigner (Sec. 2.3, 4.5)
def _gamma_matrix(N: int, sign: int, dtype=np.float64) -> np.ndarray:
    """E[k, j] = exp(sign i n_j gamma_k), n_j = j-(N-1), gamma_k = 2 pi k/(2N-1)."""
    K = 2 * N - 1
    k = np.arange(K)[:, None]
    nn = np.arange(-(N - 1), N)[None, :]
    return _expi_pi(sign * 2 * k * nn, K, dtype)


def wigner_inverse(flmn: np.ndarray, L: int, N: int, rings=None, exact: bool = False,
                   keep: bool = False) -> np.ndarray:
    """Inverse Wigner transform: f(alpha, beta, gamma) = sum (2l+1)/(8 pi^2) flmn D^{l*}_{mn}.
    ``exact``: extended-precision d-functions and sums (module docstring)."""
    dt = np.longdouble if exact else np.float64
    flmn = np.asarray(flmn).astype(_cdtype(dt))
    th = mw_thetas(L) if rings is None else mw_thetas(L)[np.asarray(rings)]
    scale = ((2 * np.arange(L).astype(np.longdouble) + 1) / (8 * PI_LD ** 2)).astype(dt)
    E = phi_dft_matrix(L, +1, dt)
    fn = []
    for j, n in enumerate(range(-(N - 1), N)):
        ft = _theta_inverse(flmn[..., j, :, :], L, n, scale, th, dt)
        fn.append(ft @ E.T)                                                  # sum_m e^{i m alpha}
    fn = np.stack(fn, axis=-3)                                               # [..., n, t, p]
    return _finish(np.einsum("kn,...ntp->...ktp", _gamma_matrix(N, +1, dt), fn), keep)   # sum_n e^{i n gamma}


def wigner_forward(f: np.ndarray, L: int, N: int, ells=None, exact: bool = False,
                   keep: bool = False) -> np.ndarray:
    """Forward Wigner transform: flmn = int f D^l_{mn}, as gamma-DFT plus spin-(-n) theta stages.
    ``exact``: extended-precision d-functions, weights and sums (module docstring)."""
    dt = np.longdouble if exact else np.float64
    f = np.asarray(f).astype(_cdtype(dt))
    if ells is None:
        ells = np.arange(L)
    qgam = (2 * PI_LD / (2 * N - 1)).astype(dt)
    fn = np.einsum("kn,...ktp->...ntp", _gamma_matrix(N, -1, dt), f) * qgam # f_n(alpha, beta)
    coef, up = _upsample_matrices(L, dt)
    ones = np.ones(L, dtype=dt)
    out = []
    for j, n in enumerate(range(-(N - 1), N)):
        G = _extend(_phi_forward(fn[..., j, :, :], L, None, dt), L, n)
        out.append(_theta_forward_upsampled(up @ (coef @ G), L, n, ones, ells, None, dt))
    return _finish(np.stack(out, axis=-3), keep)


def wigner_inverse_s(flmn: np.ndarray, L: int, N: int, sampling: str = "mw") -> np.ndarray:
    """Inverse Wigner transform on any of the samplings: for each n the spin-(-n) inverse theta
    and phi sums at that grid's (beta_t, alpha_p) with the factor (2l+1)/(8 pi^2), then the sum
    over n against e^{i n gamma_k}."""
    if sampling == "mw":
        return wigner_inverse(flmn, L, N)
    flmn = np.asarray(flmn, dtype=np.complex128)
    th = sampling_thetas(L, sampling)
    E = _phi_matrix(L, sampling_shape(L, sampling)[1], +1)
    scale = (2 * np.arange(L) + 1) / (8 * np.pi ** 2)
    fn = np.stack([_theta_inverse(flmn[..., j, :, :], L, n, scale, th) @ E.T
                   for j, n in enumerate(range(-(N - 1), N))], axis=-3)
    return np.einsum("kn,...ntp->...ktp", _gamma_matrix(N, +1), fn)


def wigner_forward_s(f: np.ndarray, L: int, N: int, sampling: str = "mw") -> np.ndarray:
    """Forward Wigner transform on any of the samplings: the gamma DFT (times 2 pi/(2N-1)), then
    for each n the theta quadrature of the sampling with d^l_{m,n} and factor 1."""
    if sampling == "mw":
        return wigner_forward(f, L, N)
    f = np.asarray(f, dtype=np.complex128)
    qgam = 2 * np.pi / (2 * N - 1)
    fn = np.einsum("kn,...ktp->...ntp", _gamma_matrix(N, -1), f) * qgam
    ones = np.ones(L)
    return np.stack([_forward_sampled(fn[..., j, :, :], L, n, ones, sampling, np.arange(L))
                     for j, n in enumerate(range(-(N - 1), N))], axis=-3)
