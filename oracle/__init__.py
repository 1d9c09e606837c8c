"""CPU oracle for the spin spherical-harmonic and Wigner transforms of Price & McEwen,
"Differentiable and accelerated spherical harmonic and Wigner transforms" (arXiv:2311.14670).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The GPU library
(``paper_2311_14670_gb300``) never imports it, and it imports nothing from the GPU library:
the two share no code.

It is plain, slow and meant to be read against the paper:

* ``sampling``   -- McEwen-Wiaux (MW) sample positions (Sec. 4.2.2) and the MW quadrature
                    weights at an upsampled bandlimit (Sec. 4.2.2, weight formula and upsampling).
* ``wigner``     -- Wigner small-d functions: the Jacobi-polynomial representation (Sec. 3.1)
                    in arbitrary precision, the paper's recursion over the order m
                    (Sec. 3.3, Eq. "wigner-d-recursion", started from Eq. "initial_values",
                    with the running renormalisation of Sec. 3.4; poles from Sec. 3.3), and, as
                    a third independent method, the half-integer recursion over the degree
                    (after Risbo 1996) from the product of representations.
* ``transforms`` -- forward / inverse spin-s SHT by separation of variables (Sec. 4.1,
                    Eqs. disc_sh_expanded, disc_sh_fft, disc_ish_fft, disc_ish_expanded) with
                    direct DFT sums, the Wigner transform as gamma-DFT plus spin-(-n) SHTs
                    (Sec. 2.3 and 4.5) and the adjoints (Sec. 5.2) as conjugate transposes.

Arithmetic is IEEE float64 except where the paper's own prescription (log-space seeds of
Eq. "initial_values") would lose accuracy in float64; there the log is taken in numpy's
extended precision (``np.longdouble``).  Every function that has no independent pin says
"parity unpinned" in its docstring; at present all are pinned by ``tests/test_oracle_*.py``.
"""
