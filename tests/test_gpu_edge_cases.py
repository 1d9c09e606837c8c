"""Degenerate cases of the method against the oracle: the largest spin a bandlimit allows
(|s| = L - 1, where only the degree l = L - 1 survives), the full azimuthal bandlimit of the Wigner
transform (N = L, so n reaches L - 1), and an empty batch, which the boundary rejects."""
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


@pytest.mark.parametrize("L,spin", [(9, 8), (40, -39)])
def test_largest_spin_matches_oracle(L, spin):
    from paper_2311_14670_gb300 import Plan
    p = Plan(L, spin=spin, max_batch=2)
    flm = synth.flm_gaussian(L, spin, 2, seed=800 + L)
    assert np.count_nonzero(flm[:, :L - 1]) == 0                # only l = L - 1 is valid
    assert rel_max(to_np(p.inverse(to_gpu(flm))), OT.inverse(flm, L, spin)) <= TOL64
    f = synth.signal_gaussian((2, L, 2 * L - 1), seed=900 + L)
    assert rel_max(to_np(p.forward(to_gpu(f))), OT.forward(f, L, spin)) <= TOL64


@pytest.mark.parametrize("L", [2, 6])
def test_wigner_full_azimuthal_bandlimit_matches_oracle(L):
    from paper_2311_14670_gb300 import Plan
    N = L
    p = Plan(L, N=N, max_batch=2)
    flmn = synth.flmn_gaussian(L, N, 2, seed=1000 + L)
    assert rel_max(to_np(p.inverse(to_gpu(flmn))), OT.wigner_inverse(flmn, L, N)) <= TOL64
    f = synth.signal_gaussian((2, 2 * N - 1, L, 2 * L - 1), seed=1100 + L)
    assert rel_max(to_np(p.forward(to_gpu(f))), OT.wigner_forward(f, L, N)) <= TOL64
    assert rel_max(to_np(p.forward(p.inverse(to_gpu(flmn)))), flmn) <= TOL64


def test_empty_batch_is_rejected():
    from paper_2311_14670_gb300 import Plan
    from paper_2311_14670_gb300 import _native as nat
    L = 8
    p = Plan(L, max_batch=2)
    x = to_gpu(synth.flm_gaussian(L, 0, 1, seed=5))
    out = torch.empty((1, L, 2 * L - 1), dtype=x.dtype, device=x.device)
    ws = p.workspace(1)
    with pytest.raises(nat.S2GBError) as e:
        nat.inverse(p._h, x, out, 0, ws, ws.numel(), 0)             # batch 0 at the C ABI
    assert e.value.code == nat.S2GB_EINVAL
    with pytest.raises(ValueError):
        p.inverse(x[:0])                                            # empty tensor in Python
    torch.cuda.synchronize()
