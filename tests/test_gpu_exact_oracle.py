"""The CUDA path against the oracle's extended-precision mode (``exact=True``: d-functions,
weights and sums in np.longdouble) on the small sphere workload (L = 64, spin 0, MW sampling), a
spin-2 batch, MWSS and DH plans and a small Wigner transform: every output element, relative max error <= 1e-12, the
float64 bar.  The float64 oracle and the extended one agree to float64 rounding (pinned in
tests/test_oracle_exact.py), so this checks the GPU against the better-conditioned reference."""
import numpy as np
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
from oracle import transforms as OT
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


@pytest.mark.parametrize("L,spin,B", [(64, 0, 1), (32, 2, 2)])
def test_sphere_inverse_and_forward_match_extended_oracle(L, spin, B):
    from paper_2311_14670_gb300 import Plan
    p = Plan(L, spin=spin, max_batch=B)
    flm = synth.flm_gaussian(L, spin, B, seed=L + B)
    f = to_np(p.inverse(to_gpu(flm)))
    ref = np.stack([OT.inverse(flm[b], L, spin, exact=True) for b in range(B)])
    assert rel_max(f, ref) <= TOL64
    rng = np.random.default_rng(L)
    g = rng.standard_normal((B, L, 2 * L - 1)) + 1j * rng.standard_normal((B, L, 2 * L - 1))
    got = to_np(p.forward(to_gpu(g)))
    ref = np.stack([OT.forward(g[b], L, spin, exact=True) for b in range(B)])
    mask = OT.coeff_mask(L, -spin)
    assert rel_max(np.where(mask, got, 0), ref) <= TOL64


@pytest.mark.parametrize("sampling", ["mwss", "dh"])
def test_samplings_match_extended_oracle(sampling):
    from paper_2311_14670_gb300 import Plan
    L, spin, B = 24, 1, 2
    p = Plan(L, spin=spin, max_batch=B, sampling=sampling)
    flm = synth.flm_gaussian(L, spin, B, seed=31)
    f = to_np(p.inverse(to_gpu(flm)))
    ref = np.stack([OT.inverse_s(flm[b], L, spin, sampling, exact=True) for b in range(B)])
    assert rel_max(f, ref) <= TOL64
    back = to_np(p.forward(to_gpu(f)))
    ref = np.stack([OT.forward_s(f[b], L, spin, sampling, exact=True) for b in range(B)])
    assert rel_max(back, ref) <= TOL64


def test_wigner_matches_extended_oracle():
    from paper_2311_14670_gb300 import Plan
    L, N = 12, 3
    p = Plan(L, N=N)
    flmn = synth.flmn_gaussian(L, N, 1, seed=9)
    f = to_np(p.inverse(to_gpu(flmn)))
    ref = OT.wigner_inverse(flmn[0], L, N, exact=True)
    assert rel_max(f[0], ref) <= TOL64
    back = to_np(p.forward(to_gpu(f)))
    ref = OT.wigner_forward(f[0], L, N, exact=True)
    assert rel_max(back[0], ref) <= TOL64
