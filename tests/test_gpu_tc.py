"""The float64 inverse theta stage with its contraction on the tensor cores (exact base-256 digit
splitting, float32 accumulation of integer digit products), against the oracle and against the
same stage on the float64 FMA pipe (S2GB_PLAN_FMA_CONTRACTION).

Bar: relative max error <= 1e-12 against the oracle; the round-trip error of the bench workload
within twice that of the FMA-pipe kernels; the device status word stays 0 (no bounded wait ran
out); results are bitwise repeatable.
"""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
from oracle import transforms as OT
from oracle.sampling import mw_thetas
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


def plans(L, spin=0, N=0, max_batch=1, **kw):
    from paper_2311_14670_gb300 import Plan
    return (Plan(L, spin=spin, N=N, max_batch=max_batch, **kw),
            Plan(L, spin=spin, N=N, max_batch=max_batch, fma_contraction=True, **kw))


def status_ok():
    from paper_2311_14670_gb300 import _native as nat
    torch.cuda.synchronize()
    return nat.device_status(torch.cuda.current_device()) == 0


# ragged ring tiles (L not a multiple of 128), degree chunks (L - l0 not a multiple of 16), the
# paired (spin 0) and unpaired slot layouts, 1 to 5 signals (1, 2 and 4 signal slots per CTA)
@pytest.mark.parametrize("L,spin,batch", [(1, 0, 1), (2, 1, 2), (5, 0, 3), (17, -3, 1), (33, 2, 5),
                                          (64, 0, 2), (129, 1, 4), (130, 0, 1), (257, -2, 3)])
def test_tc_inverse_theta_matches_oracle_and_fma(L, spin, batch):
    tc, fma = plans(L, spin, max_batch=batch)
    flm = synth.flm_gaussian(L, spin, batch, seed=9000 + L)
    x = to_gpu(flm)
    got = to_np(tc.inverse_theta(x))
    ref = OT._theta_inverse(flm, L, -spin, OT.ell_factor(L, spin), mw_thetas(L))
    T = 2 * L - 1
    perm = [(k if k <= L - 1 else k - T) + L - 1 for k in range(T)]
    assert rel_max(got, ref[..., perm]) <= TOL64
    assert rel_max(got, to_np(fma.inverse_theta(x))) <= TOL64
    assert status_ok()


@pytest.mark.parametrize("scale", [1e-250, 1e250])
def test_tc_inverse_extreme_coefficient_magnitudes(scale):
    """The per-column exponents follow the data: uniformly tiny or huge coefficients give the
    same relative error."""
    L, spin = 40, 1
    tc, _ = plans(L, spin)
    flm = synth.flm_gaussian(L, spin, 1, seed=11) * scale
    got = to_np(tc.inverse(to_gpu(flm)))
    ref = OT.inverse(flm, L, spin)
    assert rel_max(got, ref) <= TOL64
    assert status_ok()


def test_tc_inverse_column_with_wide_dynamic_range():
    """One order's coefficients spanning 2^-60 .. 1: the small ones lose bits only relative to
    the column's largest, which is what the relative max error measures."""
    L, spin = 64, 0
    tc, fma = plans(L, spin)
    flm = synth.flm_gaussian(L, spin, 1, seed=12)
    flm *= np.exp2(-np.arange(L) * 60.0 / L)[None, :, None]
    x = to_gpu(flm)
    got = to_np(tc.inverse(x))
    assert rel_max(got, OT.inverse(flm, L, spin)) <= TOL64
    assert rel_max(got, to_np(fma.inverse(x))) <= TOL64


@pytest.mark.parametrize("kind", ["wigner", "real", "mwss", "dh"])
def test_tc_inverse_other_plan_kinds(kind):
    from paper_2311_14670_gb300 import Plan
    L = 33
    if kind == "wigner":
        N = 4
        p = Plan(L, N=N, max_batch=2)
        c = synth.flmn_gaussian(L, N, 2, seed=13)
        ref = OT.wigner_inverse(c, L, N)
    elif kind == "real":
        p = Plan(L, real=True, max_batch=2)
        c = synth.flm_real_gaussian(L, 2, seed=14)
        ref = OT.inverse_real(c, L)
    else:
        p = Plan(L, spin=2, max_batch=2, sampling=kind)
        c = synth.flm_gaussian(L, 2, 2, seed=15)
        ref = OT.inverse_s(c, L, 2, kind)
    got = to_np(p.inverse(to_gpu(c)))
    assert rel_max(got, ref) <= TOL64
    assert status_ok()


def test_tc_bench_workload_round_trip_and_agreement_with_fma():
    """L = 1024, spin 2, batch 4 (coefficients complex Gaussian / (l+1)): the tensor-core inverse
    agrees with the FMA-pipe inverse to 1e-13 and the round trip is as accurate."""
    L, spin, B = 1024, 2, 4
    tc, fma = plans(L, spin, max_batch=B)
    flm = synth.flm_gaussian(L, spin, B, seed=2003, ell_power=1.0)
    x = to_gpu(flm)
    f_tc, f_fma = tc.inverse(x), fma.inverse(x)
    assert rel_max(to_np(f_tc), to_np(f_fma)) <= 1e-13
    err_tc = rel_max(to_np(tc.forward(f_tc)), flm)
    err_fma = rel_max(to_np(fma.forward(f_fma)), flm)
    assert err_tc <= max(2 * err_fma, 1e-15)
    assert torch.equal(f_tc, tc.inverse(x))              # bitwise repeatable
    assert status_ok()


@pytest.mark.parametrize("L,spin", [(1024, 2), (2048, 2), (2048, 0)])
def test_tc_flat_spectrum_round_trip_as_accurate_as_fma(L, spin):
    """Coefficients of equal variance at every degree: the low orders' ring spectra peak at the
    poles, where the theta-direction operator's diagonal is small.  With the diagonal applied in
    float64 and only the off-diagonal part on the tensor cores, the forward of the tensor-core plan
    agrees with the FMA-pipe plan's and the round trip is within twice its error."""
    tc, fma = plans(L, spin)
    flm = synth.flm_gaussian(L, spin, 1, seed=2048 + spin, ell_power=0.0)
    x = to_gpu(flm)
    f = fma.inverse(x)
    assert rel_max(to_np(tc.forward(f)), to_np(fma.forward(f))) <= 5e-14
    err_tc = rel_max(to_np(tc.forward(tc.inverse(x))), flm)
    err_fma = rel_max(to_np(fma.forward(f)), flm)
    assert err_tc <= 2 * err_fma
    assert status_ok()


def test_tc_more_than_1024_degrees_per_order():
    """L = 1500: more than 1024 degrees per order (the accumulators are read back every 128
    degrees into exact 64-bit sums), against the oracle and the FMA pipe."""
    L, spin = 1500, 1
    tc, fma = plans(L, spin)
    flm = synth.flm_gaussian(L, spin, 1, seed=16, ell_power=1.0)
    x = to_gpu(flm)
    f = tc.inverse(x)
    rings = [0, 700, 1499]
    ref = OT.inverse(flm, L, spin, rings=rings)
    assert rel_max(to_np(f)[:, rings], ref) <= TOL64
    assert rel_max(to_np(f), to_np(fma.inverse(x))) <= 1e-13
    assert status_ok()


# ---- the forward theta stage: the contraction over the rings, summed over a cluster of tiles
@pytest.mark.parametrize("L,spin,batch", [(1, 0, 1), (2, 1, 2), (5, 0, 3), (17, -3, 1), (33, 2, 5),
                                          (64, 0, 2), (129, 1, 4), (130, 0, 1), (257, -2, 3)])
def test_tc_forward_theta_matches_oracle_and_fma(L, spin, batch):
    from oracle.wigner import wigner_d_table
    tc, fma = plans(L, spin, max_batch=batch)
    g = synth.signal_gaussian((batch, 2 * L - 1, L), seed=9100 + L)
    x = to_gpu(g)
    got = to_np(tc.forward_theta(x))
    D = wigner_d_table(np.arange(L), -spin, mw_thetas(L))
    ref = np.einsum("bmt,lmt->blm", g, D) * OT.ell_factor(L, spin)[:, None]
    ref = np.where(OT.coeff_mask(L, -spin), ref, 0)
    assert rel_max(got, ref) <= TOL64
    assert rel_max(got, to_np(fma.forward_theta(x))) <= TOL64
    assert status_ok()


@pytest.mark.parametrize("L,spin", [(16, 0), (33, -1), (64, 2), (96, 0)])
def test_tc_forward_arbitrary_samples_matches_oracle(L, spin):
    tc, _ = plans(L, spin, max_batch=2)
    f = synth.signal_gaussian((2, L, 2 * L - 1), seed=9200 + L)
    assert rel_max(to_np(tc.forward(to_gpu(f))), OT.forward(f, L, spin)) <= TOL64
    assert status_ok()


@pytest.mark.parametrize("L,spin,B", [(1024, 2, 4), (2048, 0, 1)])
def test_tc_forward_full_size_agrees_with_fma(L, spin, B):
    """The bench workload (a cluster of 4 tiles of 256 rings per order) and L = 2048 spin 0 (8
    tiles, the largest cluster): tensor-core and FMA-pipe forwards agree, and the tensor-core
    forward is bitwise repeatable."""
    tc, fma = plans(L, spin, max_batch=B)
    f = to_gpu(synth.signal_gaussian((B, L, 2 * L - 1), seed=9300 + L))
    a = tc.forward(f)
    assert rel_max(to_np(a), to_np(fma.forward(f))) <= 1e-13
    assert torch.equal(a, tc.forward(f))
    assert status_ok()


def test_tc_forward_round_trip_wigner_and_samplings():
    from paper_2311_14670_gb300 import Plan
    for kw, L in [(dict(N=3), 40), (dict(spin=1, sampling="dh"), 48), (dict(spin=-2, sampling="mwss"), 48),
                  (dict(real=True), 48)]:
        p = Plan(L, max_batch=2, **kw)
        if kw.get("N"):
            c = synth.flmn_gaussian(L, kw["N"], 2, seed=L)
        elif kw.get("real"):
            c = synth.flm_real_gaussian(L, 2, seed=L)
        else:
            c = synth.flm_gaussian(L, kw["spin"], 2, seed=L)
        back = to_np(p.forward(p.inverse(to_gpu(c))))
        assert rel_max(back, c) <= TOL64, kw
    assert status_ok()
