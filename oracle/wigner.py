"""Wigner small-d functions d^l_{mn}(beta) for the oracle (test infrastructure only).

Three evaluations that share nothing but the definition (the third, ``wigner_d_halfstep``, is
documented at its definition below):

``wigner_d_jacobi``
    The Jacobi-polynomial representation of Sec. 3.1 (Eq. "wignerd_jacobi", after Varshalovich
    Sec. 4.3.4), evaluated in arbitrary precision with mpmath.  Reading of a garbled print: the
    square-root prefactor is s!(s+mu+nu)! / ((s+mu)!(s+nu)!); the printed "(s-nu)!" is undefined
    already for d^1_{10}.

``wigner_d_table``
    The paper's own recursion over the order m (Sec. 3.3, Eq. "wigner-d-recursion")

        d^l_{m-1,n} = lambda_m a_{m-1} d^l_{m,n} - (a_{m-1}/a_m) d^l_{m+1,n},
        lambda_m = (n - m cos b) / sin b,     a_m = 2 / sqrt((l-m)(l+m+1)),

    started at m = l from the closed form of Eq. "initial_values" evaluated in log space, with
    d^l_{l+1,n} = 0, and with the running (every-step) renormalisation of Sec. 3.4.  Poles use the
    closed forms d(0) = delta_{mn}, d(pi) = (-1)^{l+m} delta_{m,-n} of Sec. 3.3.

    Readings (the paper is silent on these points):
    * The running normaliser is the power of two nearest the larger magnitude of the two live
      iterates, so renormalising is exact and never divides by a zero of the oscillating iterate.
    * The log-space seed is evaluated in numpy's extended precision: in float64 the exponential of
      a logarithm of magnitude |x| carries a relative error of about eps*|x|, which reaches 1e-12
      for l ~ 2000 near the poles.  The exponent is then carried exactly as a power of two.
    * A single descending chain from m = l to m = -l leaves the oscillatory region through its lower
      turning point, where the wanted solution decays and rounding errors grow.  The recursion is
      therefore run two-sided: chain A at beta for m >= m* = round(n cos beta) (the middle of the
      oscillatory region), chain B at pi - beta for the rest, through the exact symmetry
      d^l_{m,n}(beta) = (-1)^{l+n} d^l_{-m,n}(pi - beta).  Each chain only descends from a
      forbidden region into the oscillatory one.
"""
from __future__ import annotations

import numpy as np

PI_LD = np.longdouble("3.14159265358979323846264338327950288419716939937510582097494459")
LN2_LD = np.longdouble("0.69314718055994530941723212145817656807550013436025525412068000949")


def wigner_d_jacobi(ell: int, m: int, n: int, beta, dps: int = 60):
    """d^ell_{mn}(beta) from the Jacobi-polynomial representation (Sec. 3.1), as an mpmath mpf.

    ``beta`` may be a float, a string or an mpmath number.  Returns 0 outside |m|,|n| <= ell.
    """
    import mpmath

    if abs(m) > ell or abs(n) > ell:
        return mpmath.mpf(0)
    with mpmath.workdps(dps):
        mu = abs(m - n)
        nu = abs(m + n)
        s = ell - (mu + nu) // 2
        zeta = 1 if n >= m else (-1) ** (n - m)
        f = mpmath.factorial
        pref = mpmath.sqrt(f(s) * f(s + mu + nu) / (f(s + mu) * f(s + nu)))
        b = mpmath.mpf(beta)
        val = (zeta * pref * mpmath.sin(b / 2) ** mu * mpmath.cos(b / 2) ** nu
               * mpmath.jacobi(s, mu, nu, mpmath.cos(b)))
        return +val


def _log_factorials(kmax: int) -> np.ndarray:
    """ln(k!) for k = 0..kmax in extended precision: compensated (Neumaier) running sum of ln j.

    A plain running sum would lose ~1e-14 absolute at k ~ 4000, i.e. a 1e-14 relative error in
    every seed."""
    logs = np.log(np.arange(1, kmax + 1, dtype=np.longdouble))
    out = np.zeros(kmax + 1, dtype=np.longdouble)
    s = np.longdouble(0)
    c = np.longdouble(0)
    for k in range(1, kmax + 1):
        x = logs[k - 1]
        t = s + x
        c += (s - t) + x if abs(s) >= abs(x) else (x - t) + s
        s = t
        out[k] = s + c
    return out


def _descending_chain(ells: np.ndarray, n: int, b: np.ndarray, m_stop: np.ndarray, width: int,
                      dtype=np.float64) -> np.ndarray:
    """Run Eq. "wigner-d-recursion" downward in m for every ell and angle b (0 < b < pi).

    ells: (nl,) ints with ell >= |n|.  b: (nb,) longdouble.  m_stop: (nl, nb) lowest m kept.
    Returns V of shape (nl, 2*width+1, nb) with V[i, m+width, j] = d^{ell_i}_{m,n}(b_j) for
    m_stop[i,j] <= m <= ell_i and 0 elsewhere.  ``dtype`` is the arithmetic of the recursion
    (float64, or np.longdouble for the extended-precision mode); the seeds are always evaluated
    in extended precision.
    """
    nl, nb = len(ells), len(b)
    out = np.zeros((nl, 2 * width + 1, nb), dtype=dtype)
    if nl == 0 or nb == 0:
        return out
    L2 = np.asarray(ells, dtype=np.int64)[:, None] * np.ones((1, nb), dtype=np.int64)  # ell, (nl, nb)

    # Seed d^l_{l,n}(b), Eq. "initial_values", in log space (extended precision).
    lf = _log_factorials(2 * int(np.max(ells)) + 1)
    half = b / 2
    log_s = np.log(np.sin(half))[None, :]
    log_c = np.log(np.cos(half))[None, :]
    logd = (np.longdouble(0.5) * (lf[2 * L2] - lf[L2 + n] - lf[L2 - n])
            + (L2 - n).astype(np.longdouble) * log_s + (L2 + n).astype(np.longdouble) * log_c)
    lg2 = logd / LN2_LD
    E = np.floor(lg2).astype(np.int64)                      # exact power-of-two part
    mant = np.exp2(lg2 - E.astype(np.longdouble)).astype(dtype)      # in [1, 2)
    sign = np.where((L2 - n) % 2 == 0, 1.0, -1.0).astype(dtype)   # (-sin(b/2))^{l-n}
    u_cur = sign * mant                                       # d_m   = u_cur * 2**E
    u_next = np.zeros_like(u_cur)                             # d_{m+1} (= 0 at m = l)

    # lambda_m = (n - m cos b)/sin b for every m in [-M, M], evaluated in extended precision and
    # rounded once.  Evaluating it in float64 from rounded cos b and sin b leaves a small bias of
    # the same sign at every step, which compounds over the l steps of a chain (to ~2e-13 in
    # sum_m d^2 at l = 2047 near the poles); rounded once, the error stays ~1e-15.
    M = int(np.max(ells))
    mm_all = np.arange(-M - 1, M + 2).astype(np.longdouble)[:, None]
    lam_table = ((np.longdouble(n) - mm_all * np.cos(b)[None, :]) / np.sin(b)[None, :]).astype(dtype)
    rows = np.arange(nl)[:, None]
    cols = np.arange(nb)[None, :]
    out[rows, L2 + width, cols] = np.where(L2 >= m_stop, np.ldexp(u_cur, E), 0.0)

    kmax = int(np.max(L2 - m_stop)) if np.any(L2 >= m_stop) else 0
    for k in range(1, kmax + 1):
        m = L2 - (k - 1)                      # current order; this step produces d_{m-1}
        live = (m - 1 >= m_stop) & (m - 1 >= -L2)
        p1 = np.where(live, (L2 - m + 1) * (L2 + m), 1).astype(np.longdouble)  # (l-m+1)(l+m)
        p0 = np.where(live, (L2 - m) * (L2 + m + 1), 0).astype(np.longdouble)  # (l-m)(l+m+1)
        a_m1 = (np.longdouble(2) / np.sqrt(p1)).astype(dtype)                   # a_{m-1}
        ratio = np.sqrt(p0 / p1).astype(dtype)                                   # a_{m-1}/a_m (0 at m=l)
        lam = lam_table[np.clip(m, -M - 1, M + 1) + M + 1, cols]                 # lambda_m
        u_new = lam * a_m1 * u_cur - ratio * u_next
        u_new = np.where(live, u_new, dtype(0))
        # running renormalisation (Sec. 3.4): rescale the live pair to unit size, exactly.
        r = np.maximum(np.abs(u_new), np.abs(u_cur))
        _, e = np.frexp(np.where(live & (r > 0), r, dtype(1)))
        e = np.where(live & (r > 0), e, 0)
        u_new = np.ldexp(u_new, -e)
        u_cur = np.ldexp(u_cur, -e)
        E = E + e
        u_next, u_cur = u_cur, u_new
        mm = np.where(live, m - 1, 0)
        vals = np.ldexp(u_cur, E)
        cur = out[rows, mm + width, cols]
        out[rows, mm + width, cols] = np.where(live, vals, cur)
    return out


def wigner_d_table(ells, n: int, betas, dtype=np.float64) -> np.ndarray:
    """d^l_{m,n}(beta) for every l in ``ells``, every |m| <= l and every beta in ``betas``.

    Returns D of shape (len(ells), 2*M+1, len(betas)) in ``dtype`` (float64, or np.longdouble for
    the extended-precision mode), M = max(ells), with D[i, m+M, j] = d^{ells[i]}_{m,n}(betas[j]);
    entries with |m| > l or l < |n| are 0.  ``betas`` in [0, pi]; pass ``np.longdouble`` values for
    full accuracy of the seeds.
    """
    ells = np.atleast_1d(np.asarray(ells, dtype=np.int64))
    betas = np.atleast_1d(np.asarray(betas)).astype(np.longdouble)
    M = int(ells.max()) if len(ells) else 0
    nl, nb = len(ells), len(betas)
    D = np.zeros((nl, 2 * M + 1, nb), dtype=dtype)
    tol = np.longdouble(8) * np.longdouble(np.finfo(np.float64).eps)
    north = betas <= tol
    south = np.abs(betas - PI_LD) <= tol
    inner = ~(north | south)
    ok = ells >= abs(n)

    # Poles, Sec. 3.3: d(0) = delta_{mn}, d(pi) = (-1)^{l+m} delta_{m,-n}.
    for i in np.nonzero(ok)[0]:
        ell = int(ells[i])
        D[i, n + M, north] = 1.0
        D[i, -n + M, south] = (-1.0) ** (ell - n)

    idx_l = np.nonzero(ok)[0]
    idx_b = np.nonzero(inner)[0]
    if len(idx_l) == 0 or len(idx_b) == 0:
        return D
    L_ok = ells[idx_l]
    b = betas[idx_b]
    # Split point m* = round(n cos beta), clipped to [-l, l] (Sec. 3.3 reading, module docstring).
    mstar = np.rint(n * np.cos(b.astype(np.float64))).astype(np.int64)[None, :]
    mstar = np.clip(mstar, -L_ok[:, None], L_ok[:, None])
    A = _descending_chain(L_ok, n, b, mstar, M, dtype)               # m in [m*, l] at beta
    B = _descending_chain(L_ok, n, PI_LD - b, 1 - mstar, M, dtype)   # m' in [1-m*, l] at pi-beta
    sgn = np.where((L_ok + n) % 2 == 0, 1.0, -1.0).astype(dtype)[:, None, None]
    B_reflected = sgn * B[:, ::-1, :]                                  # m = -m'
    mgrid = np.arange(-M, M + 1)[None, :, None]
    useA = mgrid >= mstar[:, None, :]
    blockD = np.where(useA, A, B_reflected)
    blockD = np.where(np.abs(mgrid) <= L_ok[:, None, None], blockD, dtype(0))
    D[np.ix_(idx_l, np.arange(2 * M + 1), idx_b)] = blockD
    return D


def wigner_d_halfstep(L: int, betas) -> np.ndarray:
    """d^l_{mn}(beta) for every integer l < L and all |m|, |n| <= l, by the half-integer recursion
    over the degree (after Risbo 1996): the representation of degree j is the stretched part of
    the product of those of degrees j - 1/2 and 1/2, so with the Clebsch-Gordan coefficients
    <j-1/2, m-mu; 1/2, mu | j, m> = sqrt((j + 2 mu m) / (2j)),

        d^j_{mn} = sum_{mu, nu = +-1/2} sqrt((j + 2 mu m)(j + 2 nu n)) / (2j)
                                        d^{j-1/2}_{m-mu, n-nu} d^{1/2}_{mu nu},

    d^{1/2}_{++} = d^{1/2}_{--} = cos(b/2), d^{1/2}_{+-} = -sin(b/2), d^{1/2}_{-+} = sin(b/2).
    Every step is a product of unitary maps, so the recursion is stable in float64 at any beta;
    it shares nothing with the recursion over m or the Jacobi form.  O(L^3) per angle: for test
    sizes.  Returns D of shape (L, 2L-1, 2L-1, len(betas)) with D[l, m+L-1, n+L-1, k] =
    d^l_{mn}(betas[k]) (0 where |m| or |n| > l).
    """
    b = np.atleast_1d(np.asarray(betas)).astype(np.longdouble)
    p = np.cos(b / 2).astype(np.float64)
    q = np.sin(b / 2).astype(np.float64)
    nb = len(b)
    out = np.zeros((L, 2 * L - 1, 2 * L - 1, nb))
    d = np.ones((1, 1, nb))                        # degree 0
    out[0, L - 1, L - 1] = 1.0
    for tj in range(1, 2 * L - 1):                 # 2j, j = 1/2, 1, ..., L-1
        a = np.arange(tj + 1)                      # m = -j + a
        sa = np.sqrt(a / tj)[:, None, None]        # sqrt((j + m) / (2j))
        ra = np.sqrt((tj - a) / tj)[:, None, None]  # sqrt((j - m) / (2j))
        sb = np.sqrt(a / tj)[None, :, None]
        rb = np.sqrt((tj - a) / tj)[None, :, None]
        prev = np.zeros((tj + 2, tj + 2, nb))      # padded: prev index a' + 1
        prev[1:tj + 1, 1:tj + 1] = d
        pm = prev[0:tj + 1, 0:tj + 1]              # d^{j-1/2}_{m-1/2, n-1/2}
        p_ = prev[0:tj + 1, 1:tj + 2]              # d^{j-1/2}_{m-1/2, n+1/2}
        m_ = prev[1:tj + 2, 0:tj + 1]              # d^{j-1/2}_{m+1/2, n-1/2}
        mm = prev[1:tj + 2, 1:tj + 2]              # d^{j-1/2}_{m+1/2, n+1/2}
        d = (sa * sb * p * pm - sa * rb * q * p_ + ra * sb * q * m_ + ra * rb * p * mm)
        if tj % 2 == 0:
            l = tj // 2
            out[l, L - 1 - l:L + l, L - 1 - l:L + l] = d
    return out

