"""Forward transforms at full size on arbitrary (not bandlimited) samples, against the oracle.

* The ±m-paired forward theta kernels (spin-0 plans: one recursion feeds the columns m and -m) at
  L = 1024 and L = 2048 with two signals, on sampled degrees of every order.  Round trips cannot
  check these instances: bandlimited inputs never excite the odd-parity part of the torus
  extension that arbitrary samples carry.
* Whole coefficient columns (every degree l of a few orders m) of the unpaired L = 1024, spin-2,
  batch-4 forward, so that every degree position of the per-order reduction is compared.

The oracle's d-functions cost the same per degree whichever orders are kept, so its degrees are
split over spawned host processes (`oracle_forward_parallel`).  Bar: relative max error <= 1e-12.
"""
import numpy as np
import pytest

from gpu_helpers import TOL64, oracle_forward_parallel, rel_max, to_gpu, to_np
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


@pytest.mark.parametrize("L,ells", [(1024, [0, 1, 2, 255, 512, 1000, 1022, 1023]),
                                    (2048, [0, 1, 777, 2046, 2047])])
def test_paired_forward_spin0_batch2_arbitrary_samples_sampled_degrees(L, ells):
    from paper_2311_14670_gb300 import Plan
    B = 2
    p = Plan(L, spin=0, max_batch=B)
    f = synth.signal_gaussian((B, L, 2 * L - 1), seed=3100 + L)
    got = to_np(p.forward(to_gpu(f)))
    ref = oracle_forward_parallel(f, L, 0, ells)
    assert rel_max(got[:, ells], ref) <= TOL64


def test_forward_whole_columns_L1024_spin2_batch4():
    from paper_2311_14670_gb300 import Plan
    L, spin, B = 1024, 2, 4
    orders = [0, -1, 1, 17, -17, 511, -511, L - 1]
    p = Plan(L, spin=spin, max_batch=B)
    f = synth.signal_gaussian((B, L, 2 * L - 1), seed=3200)
    got = to_np(p.forward(to_gpu(f)))
    ref = oracle_forward_parallel(f, L, spin, range(L), orders=orders)     # [b][l][orders]
    cols = [m + L - 1 for m in orders]
    assert rel_max(got[:, :, cols], ref) <= TOL64
    # the degrees below max(|m|, |s|) are zero on both sides
    for k, m in enumerate(orders):
        lo = max(abs(m), abs(spin))
        assert np.all(got[:, :lo, cols[k]] == 0) and np.all(ref[:, :lo, k] == 0)
