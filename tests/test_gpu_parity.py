"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Bar (float64): relative max error max|gpu - oracle| / max|oracle| <= 1e-12 on the same seeded
inputs.  Small cases compare every output; the full-size workloads (L = 1024 spin 2 batch 4;
L = 2048 spin 0) compare sampled rings / degrees the oracle computes one by one.
"""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
from oracle import transforms as OT
from oracle.sampling import mw_thetas
from oracle.wigner import wigner_d_table
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


def plan(L, spin=0, N=0, max_batch=1):
    from paper_2311_14670_gb300 import Plan
    return Plan(L, spin=spin, N=N, max_batch=max_batch)


SMALL = [(1, 0), (2, 0), (2, 1), (3, -2), (16, 0), (17, 3), (33, -1), (64, 2), (130, 0), (257, -3)]


@pytest.mark.parametrize("L,spin", SMALL)
@pytest.mark.parametrize("batch", [1, 3])
def test_inverse_theta_matches_oracle(L, spin, batch):
    p = plan(L, spin, max_batch=batch)
    flm = synth.flm_gaussian(L, spin, batch, seed=L * 7 + batch)
    got = to_np(p.inverse_theta(to_gpu(flm)))                             # [b][t][m mod T]
    ref = OT._theta_inverse(flm, L, -spin, OT.ell_factor(L, spin), mw_thetas(L))   # [b][t][m+L-1]
    T = 2 * L - 1
    perm = [(k if k <= L - 1 else k - T) + L - 1 for k in range(T)]
    assert rel_max(got, ref[..., perm]) <= TOL64


@pytest.mark.parametrize("L,spin", SMALL)
@pytest.mark.parametrize("batch", [1, 2, 5])
def test_forward_theta_matches_oracle(L, spin, batch):
    p = plan(L, spin, max_batch=batch)
    g = synth.signal_gaussian((batch, 2 * L - 1, L), seed=L + 11 * batch)
    got = to_np(p.forward_theta(to_gpu(g)))
    D = wigner_d_table(np.arange(L), -spin, mw_thetas(L))                 # [l][m][t]
    ref = np.einsum("bmt,lmt->blm", g, D) * OT.ell_factor(L, spin)[:, None]
    ref = np.where(OT.coeff_mask(L, -spin), ref, 0)
    assert rel_max(got, ref) <= TOL64


@pytest.mark.parametrize("L,spin", SMALL)
def test_inverse_matches_oracle(L, spin):
    batch = 2
    p = plan(L, spin, max_batch=batch)
    flm = synth.flm_gaussian(L, spin, batch, seed=100 + L)
    got = to_np(p.inverse(to_gpu(flm)))
    ref = OT.inverse(flm, L, spin)
    assert rel_max(got, ref) <= TOL64


@pytest.mark.parametrize("L,spin", [(1, 0), (2, 0), (2, 1), (3, -2), (16, 0), (17, 3), (33, -1), (64, 2), (96, 0)])
def test_forward_matches_oracle_on_arbitrary_samples(L, spin):
    """Arbitrary (not bandlimited) samples exercise the whole linear map of the forward transform."""
    batch = 2
    p = plan(L, spin, max_batch=batch)
    f = synth.signal_gaussian((batch, L, 2 * L - 1), seed=200 + L)
    got = to_np(p.forward(to_gpu(f)))
    ref = OT.forward(f, L, spin)
    assert rel_max(got, ref) <= TOL64


@pytest.mark.parametrize("L,spin", [(8, 0), (31, 1), (64, -2), (200, 0), (256, 2)])
def test_round_trip(L, spin):
    p = plan(L, spin, max_batch=2)
    flm = synth.flm_gaussian(L, spin, 2, seed=300 + L)
    x = to_gpu(flm)
    back = to_np(p.forward(p.inverse(x)))
    assert rel_max(back, flm) <= TOL64


@pytest.mark.parametrize("L,spin", [(3, 0), (9, 1), (16, -2), (40, 0)])
def test_adjoints_match_oracle(L, spin):
    batch = 2
    p = plan(L, spin, max_batch=batch)
    y = synth.signal_gaussian((batch, L, 2 * L - 1), seed=400 + L)
    got = to_np(p.adjoint_inverse(to_gpu(y)))
    assert rel_max(got, OT.adjoint_inverse(y, L, spin)) <= TOL64
    c = synth.flm_gaussian(L, spin, batch, seed=500 + L)
    got = to_np(p.adjoint_forward(to_gpu(c)))
    assert rel_max(got, OT.adjoint_forward(c, L, spin)) <= TOL64


@pytest.mark.parametrize("L,spin", [(128, 0), (333, 1)])
def test_adjoint_dot_products(L, spin):
    """<A x, y> = <x, A^H y> for both transforms at sizes beyond the dense oracle."""
    p = plan(L, spin)
    x = to_gpu(synth.flm_gaussian(L, spin, 1, seed=1))
    y = to_gpu(synth.signal_gaussian((1, L, 2 * L - 1), seed=2))
    lhs = torch.vdot(p.inverse(x).flatten(), y.flatten())
    rhs = torch.vdot(x.flatten(), p.adjoint_inverse(y).flatten())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs = torch.vdot(p.forward(y).flatten(), x.flatten())
    rhs = torch.vdot(y.flatten(), p.adjoint_forward(x).flatten())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("L,N", [(4, 1), (8, 3), (13, 4)])
def test_wigner_matches_oracle(L, N):
    batch = 2
    p = plan(L, N=N, max_batch=batch)
    flmn = synth.flmn_gaussian(L, N, batch, seed=600 + L)
    got = to_np(p.inverse(to_gpu(flmn)))
    assert rel_max(got, OT.wigner_inverse(flmn, L, N)) <= TOL64
    f = synth.signal_gaussian((batch, 2 * N - 1, L, 2 * L - 1), seed=700 + L)
    got = to_np(p.forward(to_gpu(f)))
    assert rel_max(got, OT.wigner_forward(f, L, N)) <= TOL64
    back = to_np(p.forward(p.inverse(to_gpu(flmn))))
    assert rel_max(back, flmn) <= TOL64


def test_wigner_adjoint_dot_products():
    L, N = 32, 5
    p = plan(L, N=N)
    x = to_gpu(synth.flmn_gaussian(L, N, 1, seed=3))
    y = to_gpu(synth.signal_gaussian((1, 2 * N - 1, L, 2 * L - 1), seed=4))
    lhs = torch.vdot(p.inverse(x).flatten(), y.flatten())
    rhs = torch.vdot(x.flatten(), p.adjoint_inverse(y).flatten())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs = torch.vdot(p.forward(y).flatten(), x.flatten())
    rhs = torch.vdot(y.flatten(), p.adjoint_forward(x).flatten())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_full_size_L1024_spin2_batch4_inverse_sampled_rings():
    """The bench workload: L = 1024, spin 2, batch 4, flm ~ complex Gaussian / (l+1)."""
    L, spin, B = 1024, 2, 4
    p = plan(L, spin, max_batch=B)
    flm = synth.flm_gaussian(L, spin, B, seed=2001, ell_power=1.0)
    got = to_np(p.inverse(to_gpu(flm)))
    rings = [0, 1, 2, 300, 511, 900, 1021, 1022, 1023]
    ref = OT.inverse(flm, L, spin, rings=rings)
    assert rel_max(got[:, rings], ref) <= TOL64


def test_full_size_L1024_spin2_batch4_forward_sampled_degrees():
    L, spin, B = 1024, 2, 4
    p = plan(L, spin, max_batch=B)
    f = synth.signal_gaussian((B, L, 2 * L - 1), seed=2002)
    got = to_np(p.forward(to_gpu(f)))
    ells = [2, 3, 17, 256, 511, 777, 1022, 1023]
    ref = OT.forward(f, L, spin, ells=ells)
    assert rel_max(got[:, ells], ref) <= TOL64


def test_full_size_L1024_round_trip():
    L, spin, B = 1024, 2, 4
    p = plan(L, spin, max_batch=B)
    flm = synth.flm_gaussian(L, spin, B, seed=2003, ell_power=1.0)
    back = to_np(p.forward(p.inverse(to_gpu(flm))))
    assert rel_max(back, flm) <= TOL64


def test_full_size_L2048_spin0_inverse_sampled_rings_and_round_trip():
    L = 2048
    p = plan(L, 0)
    flm = synth.flm_gaussian(L, 0, 1, seed=2004)
    x = to_gpu(flm)
    f = p.inverse(x)
    rings = [0, 1, 1023, 2046, 2047]
    ref = OT.inverse(flm, L, 0, rings=rings)
    assert rel_max(to_np(f)[:, rings], ref) <= TOL64
    back = to_np(p.forward(f))
    assert rel_max(back, flm) <= TOL64


def test_partial_batch_and_determinism():
    L, spin = 48, 1
    p = plan(L, spin, max_batch=4)
    flm = synth.flm_gaussian(L, spin, 3, seed=9)
    x = to_gpu(flm)
    a = p.inverse(x)
    b = p.inverse(x)
    assert torch.equal(a, b)                                   # deterministic
    one = torch.cat([p.inverse(x[i:i + 1]) for i in range(3)])
    assert rel_max(to_np(one), to_np(a)) <= TOL64
    fa = p.forward(a)
    assert torch.equal(fa, p.forward(a))


def test_argument_errors():
    from paper_2311_14670_gb300 import _native as nat
    L = 8
    p = plan(L, 0, max_batch=2)
    x = to_gpu(synth.flm_gaussian(L, 0, 2, seed=1))
    ws = p.workspace(2)
    with pytest.raises(nat.S2GBError) as e:
        nat.inverse(p._h, x, x, 2, ws, ws.numel(), 0)               # in == out
    assert e.value.code == nat.S2GB_EINVAL
    out = torch.empty_like(x)
    with pytest.raises(nat.S2GBError) as e:
        nat.inverse(p._h, x, out, 2, ws, 16, 0)                      # workspace too small
    assert e.value.code == nat.S2GB_EWORKSPACE
    with pytest.raises(nat.S2GBError) as e:
        nat.inverse(p._h, x, out, 3, ws, ws.numel(), 0)             # batch > max_batch
    assert e.value.code == nat.S2GB_EINVAL
    torch.cuda.synchronize()


@pytest.mark.parametrize("L,spin", [(2500, 1), (4096, 0)])
def test_beyond_2048_chunked_forward_and_sampled_parity(L, spin):
    """L > 2048: the forward theta stage runs in ring chunks (polar caps + interior) summed in a
    fixed order.  Round trip, plus sampled rings of the inverse against the oracle."""
    p = plan(L, spin)
    flm = synth.flm_gaussian(L, spin, 1, seed=L, ell_power=1.0)
    x = to_gpu(flm)
    f = p.inverse(x)
    back = to_np(p.forward(f))
    assert rel_max(back, flm) <= TOL64
    rings = [1, L // 2, L - 2]
    ref = OT.inverse(flm, L, spin, rings=rings)
    assert rel_max(to_np(f)[:, rings], ref) <= TOL64


def test_L2500_forward_sampled_degrees_on_arbitrary_samples():
    L, spin = 2500, -2
    p = plan(L, spin)
    f = synth.signal_gaussian((1, L, 2 * L - 1), seed=77)
    got = to_np(p.forward(to_gpu(f)))
    ells = [2, 1000, 2499]
    ref = OT.forward(f, L, spin, ells=ells)
    assert rel_max(got[:, ells], ref) <= TOL64


def test_L8192_round_trip():
    L = 8192
    p = plan(L, 0)
    flm = synth.flm_gaussian(L, 0, 1, seed=8192, ell_power=1.0)
    back = to_np(p.forward(p.inverse(to_gpu(flm))))
    assert rel_max(back, flm) <= TOL64


def test_kernel_launch_counter_counts_each_stage():
    """s2gb_kernels_launched counts this library's own launches: the sphere inverse is one theta
    kernel (then cuFFT); the forward is the theta-direction operator on the tensor cores (column
    exponents + the operator GEMM) plus the theta kernel, or, with the contraction on the FMA pipe,
    four glue kernels around the operator's FFTs plus the theta kernel; above L = 2048 the forward
    theta stage is several ring-chunk launches and one fixed-order sum."""
    from paper_2311_14670_gb300 import Plan
    from paper_2311_14670_gb300 import _native as nat
    x = to_gpu(synth.flm_gaussian(64, 2, 1, seed=5))
    for p, counts in [(plan(64, 2), (1, 3)), (Plan(64, spin=2, fma_contraction=True), (1, 5))]:
        k0 = nat.kernels_launched()
        f = p.inverse(x)
        k1 = nat.kernels_launched()
        p.forward(f)
        k2 = nat.kernels_launched()
        assert (k1 - k0, k2 - k1) == counts
    q = plan(2500, 0)
    g = q.inverse(to_gpu(synth.flm_gaussian(2500, 0, 1, seed=6)))
    k3 = nat.kernels_launched()
    q.forward(g)
    assert nat.kernels_launched() - k3 >= 4 + 3 + 1     # caps, >= 1 interior chunk, sum
