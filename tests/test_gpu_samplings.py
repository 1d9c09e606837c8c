"""Parity of the MWSS and DH samplings (Sec. 4.2) on the GPU with the CPU oracle.

Bar (float64): relative max error max|gpu - oracle| / max|oracle| <= 1e-12 on the same seeded
inputs.  Small cases compare every output (inverse on bandlimited coefficients, forward on
arbitrary samples, which exercises the whole linear map including the MWSS poles and the phi
frequency no order owns), adjoints against the oracle's dense conjugate transpose; large cases
compare sampled rings and round trips, including the ring-chunked forward (DH, more than 2048
rings).  On MWSS the recursion runs over the interior rings and the pole rings are exact.
"""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
from oracle import transforms as OT
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLINGS = ["mwss", "dh"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


def plan(L, sampling, spin=0, N=0, max_batch=1, precision="fp64", real=False):
    from paper_2311_14670_gb300 import Plan
    return Plan(L, spin=spin, N=N, max_batch=max_batch, sampling=sampling, precision=precision, real=real)


SMALL = [(1, 0), (2, 0), (2, 1), (3, -2), (16, 0), (17, 3), (33, -1), (64, 2), (130, 0)]


@pytest.mark.parametrize("sampling", SAMPLINGS)
@pytest.mark.parametrize("L,spin", SMALL)
def test_inverse_matches_oracle(sampling, L, spin):
    batch = 2
    p = plan(L, sampling, spin, max_batch=batch)
    flm = synth.flm_gaussian(L, spin, batch, seed=700 + L)
    got = to_np(p.inverse(to_gpu(flm)))
    ref = OT.inverse_s(flm, L, spin, sampling)
    assert got.shape == ref.shape
    assert rel_max(got, ref) <= TOL64


@pytest.mark.parametrize("sampling", SAMPLINGS)
@pytest.mark.parametrize("L,spin", [(1, 0), (2, 0), (2, 1), (3, -2), (16, 0), (17, 3), (33, -1), (64, 2)])
def test_forward_matches_oracle_on_arbitrary_samples(sampling, L, spin):
    batch = 2
    p = plan(L, sampling, spin, max_batch=batch)
    R, P = OT.sampling_shape(L, sampling)
    f = synth.signal_gaussian((batch, R, P), seed=800 + L)
    got = to_np(p.forward(to_gpu(f)))
    ref = OT.forward_s(f, L, spin, sampling)
    assert rel_max(got, ref) <= TOL64


@pytest.mark.parametrize("sampling", SAMPLINGS)
@pytest.mark.parametrize("L,spin", [(8, 0), (31, 1), (200, -2), (256, 0)])
def test_round_trip(sampling, L, spin):
    p = plan(L, sampling, spin, max_batch=2)
    flm = synth.flm_gaussian(L, spin, 2, seed=900 + L)
    back = to_np(p.forward(p.inverse(to_gpu(flm))))
    assert rel_max(back, flm) <= TOL64


@pytest.mark.parametrize("sampling", SAMPLINGS)
@pytest.mark.parametrize("L,spin", [(2, 0), (3, 1), (5, -2)])
def test_adjoints_match_dense_oracle(sampling, L, spin):
    """The adjoints equal the conjugate transposes of the oracle's linear maps, built column by
    column from unit vectors."""
    p = plan(L, sampling, spin)
    R, P = OT.sampling_shape(L, sampling)
    y = synth.signal_gaussian((R, P), seed=L + 1)
    ref = OT.adjoint_dense(lambda x: OT.inverse_s(x, L, spin, sampling), (L, 2 * L - 1), y)
    ref = np.where(OT.coeff_mask(L, -spin), ref, 0)
    got = to_np(p.adjoint_inverse(to_gpu(y[None])))[0]
    assert rel_max(got, ref) <= TOL64
    c = synth.flm_gaussian(L, spin, 1, seed=L + 2)[0]
    ref = OT.adjoint_dense(lambda x: OT.forward_s(x, L, spin, sampling), (R, P), c)
    got = to_np(p.adjoint_forward(to_gpu(c[None])))[0]
    assert rel_max(got, ref) <= TOL64


@pytest.mark.parametrize("sampling", SAMPLINGS)
@pytest.mark.parametrize("L,spin", [(128, 0), (333, 1)])
def test_adjoint_dot_products(sampling, L, spin):
    p = plan(L, sampling, spin)
    R, P = OT.sampling_shape(L, sampling)
    x = to_gpu(synth.flm_gaussian(L, spin, 1, seed=3))
    y = to_gpu(synth.signal_gaussian((1, R, P), seed=4))
    lhs = torch.vdot(p.inverse(x).flatten(), y.flatten())
    rhs = torch.vdot(x.flatten(), p.adjoint_inverse(y).flatten())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs = torch.vdot(p.forward(y).flatten(), x.flatten())
    rhs = torch.vdot(y.flatten(), p.adjoint_forward(x).flatten())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("sampling", SAMPLINGS)
@pytest.mark.parametrize("L,N", [(4, 1), (8, 3), (13, 4)])
def test_wigner_matches_oracle(sampling, L, N):
    batch = 2
    p = plan(L, sampling, N=N, max_batch=batch)
    flmn = synth.flmn_gaussian(L, N, batch, seed=1000 + L)
    got = to_np(p.inverse(to_gpu(flmn)))
    ref = OT.wigner_inverse_s(flmn, L, N, sampling)
    assert rel_max(got, ref) <= TOL64
    R, P = OT.sampling_shape(L, sampling)
    f = synth.signal_gaussian((batch, 2 * N - 1, R, P), seed=1100 + L)
    assert rel_max(to_np(p.forward(to_gpu(f))), OT.wigner_forward_s(f, L, N, sampling)) <= TOL64
    assert rel_max(to_np(p.forward(p.inverse(to_gpu(flmn)))), flmn) <= TOL64


@pytest.mark.parametrize("L", [2, 9, 64, 257])
def test_dh_real_signals_match_oracle(L):
    batch = 2
    p = plan(L, "dh", max_batch=batch, real=True)
    a = synth.flm_gaussian(L, 0, batch, seed=1200 + L)[..., L - 1:]       # orders m >= 0
    got = to_np(p.inverse(to_gpu(a)))
    ref = OT.inverse_real(a, L, "dh")
    assert rel_max(got, ref) <= TOL64
    f = synth.signal_gaussian((batch, 2 * L, 2 * L - 1), seed=1300 + L).real.copy()
    assert rel_max(to_np(p.forward(to_gpu(f))), OT.forward_real(f, L, "dh")) <= TOL64


def test_real_mwss_is_refused():
    from paper_2311_14670_gb300 import _native as nat
    with pytest.raises(nat.S2GBError) as e:
        plan(8, "mwss", real=True)
    assert e.value.code == nat.S2GB_EUNSUPPORTED


@pytest.mark.parametrize("sampling,L,spin,batch,rings", [
    ("dh", 1024, 2, 2, [0, 1, 5, 700, 1023, 1024, 1500, 2046, 2047]),
    ("mwss", 1024, 2, 2, [0, 1, 2, 512, 1000, 1022, 1023, 1024]),
    ("mwss", 2048, 0, 1, [0, 1, 3, 1024, 2047, 2048]),
])
def test_large_sampled_rings_and_round_trip(sampling, L, spin, batch, rings):
    """Full-size cases: sampled rings of the inverse against the oracle (the MWSS poles among
    them), and the round trip."""
    p = plan(L, sampling, spin, max_batch=batch)
    flm = synth.flm_gaussian(L, spin, batch, seed=1400 + L)
    x = to_gpu(flm)
    f = p.inverse(x)
    got = to_np(f[:, rings])
    ref = OT.inverse_s(flm, L, spin, sampling, rings=rings)
    assert rel_max(got, ref) <= TOL64
    back = to_np(p.forward(f))
    assert rel_max(back, flm) <= TOL64


def test_dh_ring_chunked_forward():
    """DH at L = 1100 has 2200 rings: the forward theta stage runs in ring chunks (polar caps and
    interior) summed in a fixed order; compare sampled degrees with the oracle on arbitrary samples."""
    L, spin = 1100, 1
    p = plan(L, "dh", spin)
    f = synth.signal_gaussian((1, 2 * L, 2 * L - 1), seed=5)
    got = to_np(p.forward(to_gpu(f)))
    ells = np.array([1, 2, 50, 333, 700, 1098, 1099])
    ref = OT.forward_s(f, L, spin, "dh", ells=ells)
    assert rel_max(got[:, ells], ref) <= TOL64


@pytest.mark.parametrize("sampling", SAMPLINGS)
@pytest.mark.parametrize("L,spin", [(64, 0), (256, 2)])
def test_fp32_plans_against_fp64(sampling, L, spin):
    """Float32 plans on the other samplings: error against the float64 path of the same GPU, at the
    level the MW float32 path reaches (relative max error below 1e-5)."""
    batch = 2
    p64 = plan(L, sampling, spin, max_batch=batch)
    p32 = plan(L, sampling, spin, max_batch=batch, precision="fp32")
    flm = synth.flm_gaussian(L, spin, batch, seed=1500 + L)
    f64 = p64.inverse(to_gpu(flm))
    f32 = p32.inverse(to_gpu(flm, torch.complex64))
    assert rel_max(to_np(f32), to_np(f64)) <= 1e-5
    b64 = p64.forward(f64)
    b32 = p32.forward(f64.to(torch.complex64))
    assert rel_max(to_np(b32), to_np(b64)) <= 1e-5


@pytest.mark.parametrize("sampling", SAMPLINGS)
def test_order_sharded_transforms_are_bitwise_unsharded(sampling):
    """Sequential |m|-range shards assemble to the unsharded transforms bit for bit (the MWSS ring
    spectra carry the column k = L, which every shard writes as 0)."""
    from paper_2311_14670_gb300.multigpu import column_owner, order_ranges
    L, spin, batch, world = 40, 1, 2, 3
    p = plan(L, sampling, spin, max_batch=batch)
    flm = to_gpu(synth.flm_gaussian(L, spin, batch, seed=6))
    R, P = OT.sampling_shape(L, sampling)
    f = to_gpu(synth.signal_gaussian((batch, R, P), seed=7))
    ranges = order_ranges(L, world, abs(spin))
    ft = torch.full(p.spectra_shape(batch), 7.0 + 1j, dtype=p.dtype, device=p.device)
    fl = torch.zeros(p.coef_shape(batch), dtype=p.dtype, device=p.device)
    for lo, hi in ranges:
        p.inverse_theta_mrange(flm, lo, hi, out=ft)
        p.forward_mrange(f, lo, hi, out=fl)
    assert column_owner(L, ranges, "mod", P)[L % P] >= 0
    assert torch.equal(p.inverse_phi(ft), p.inverse(flm))
    assert torch.equal(fl, p.forward(f))


@pytest.mark.parametrize("L,spin,batch", [(1, 0, 1), (2, 1, 2), (5, -2, 3), (40, 0, 2), (97, 3, 1)])
def test_mwss_theta_stages_include_the_poles(L, spin, batch):
    """The theta stages alone on MWSS: the recursion covers the interior rings and the pole rings
    theta = 0, pi (Kronecker-delta d-functions) are added exactly; both compared with the oracle's
    d-functions on all L+1 rings."""
    from oracle.sampling import mwss_thetas
    from oracle.wigner import wigner_d_table
    p = plan(L, "mwss", spin, max_batch=batch)
    flm = synth.flm_gaussian(L, spin, batch, seed=L + 40)
    got = to_np(p.inverse_theta(to_gpu(flm)))                             # [b][t][m mod 2L]
    ref = OT._theta_inverse(flm, L, -spin, OT.ell_factor(L, spin), mwss_thetas(L))
    cols = [m % (2 * L) for m in range(-(L - 1), L)]
    assert rel_max(got[..., cols], ref) <= TOL64
    assert np.all(got[..., L] == 0)                                       # the phi frequency L
    g = synth.signal_gaussian((batch, 2 * L - 1, L + 1), seed=L + 41)
    D = wigner_d_table(np.arange(L), -spin, mwss_thetas(L))               # [l][m][t]
    ref = np.einsum("bmt,lmt->blm", g, D) * OT.ell_factor(L, spin)[:, None]
    ref = np.where(OT.coeff_mask(L, -spin), ref, 0)
    assert rel_max(to_np(p.forward_theta(to_gpu(g))), ref) <= TOL64
