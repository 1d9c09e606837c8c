"""The allocation-free inverse transform (s2gb_inverse_noalloc) gives the same results as
s2gb_inverse.

It is for callers that cannot allocate device memory where they run the transform (memory owned by
another allocator, no-allocation rules, plugins handed only their input and output), so it works
from a static device array inside libs2gb.so.  Two calls in a row check that the array's left-over
contents from the previous call do not leak into the next result.  This file is collected last so
that a failure here leaves every other test already run.
"""
import pytest

from gpu_helpers import TOL64, rel_max, to_gpu, to_np
from paper_2311_14670_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    from paper_2311_14670_gb300 import build
    build.build()


# (L, spin, N, batch, max_batch, precision): sphere and Wigner plans, full and partial batches
# (a partial Wigner batch runs its gamma DFT signal by signal), float64 and float32
CASES = [(64, 1, 0, 3, 3, "fp64"), (130, -2, 0, 2, 4, "fp64"), (12, 0, 3, 2, 2, "fp64"),
         (12, 0, 3, 1, 3, "fp64"), (64, 2, 0, 2, 2, "fp32"), (20, 0, 2, 1, 2, "fp32")]


@pytest.mark.parametrize("L,spin,N,batch,max_batch,precision", CASES)
def test_noalloc_inverse_matches_inverse_on_two_calls(L, spin, N, batch, max_batch, precision):
    from paper_2311_14670_gb300 import Plan
    from paper_2311_14670_gb300 import _native as nat

    plan = Plan(L, spin=spin, N=N, max_batch=max_batch, precision=precision)
    # the same stages and kernels as s2gb_inverse, so float32 agrees to its own rounding level
    tol = TOL64 if precision == "fp64" else 1e-6
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        seed = 10 * call + L
        coef = synth.flmn_gaussian(L, N, batch, seed) if N else synth.flm_gaussian(L, spin, batch, seed)
        x = to_gpu(coef, plan.dtype)
        ref = plan.inverse(x)
        out = torch.full_like(ref, float("nan"))
        nat.inverse_noalloc(plan._h, x, out, batch, stream)
        torch.cuda.synchronize()
        assert rel_max(to_np(out), to_np(ref)) <= tol


def test_noalloc_inverse_allocates_nothing():
    """After a first call on the device, further calls change neither the device's free memory nor
    the bytes held by PyTorch's allocator."""
    from paper_2311_14670_gb300 import Plan
    from paper_2311_14670_gb300 import _native as nat

    L, spin, B = 96, 2, 2
    plan = Plan(L, spin=spin, max_batch=B)
    x = to_gpu(synth.flm_gaussian(L, spin, B, seed=5))
    out = torch.empty(plan.shape(B), dtype=plan.signal_dtype, device=x.device)
    stream = torch.cuda.current_stream().cuda_stream
    nat.inverse_noalloc(plan._h, x, out, B, stream)
    torch.cuda.synchronize()
    free0, held0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        nat.inverse_noalloc(plan._h, x, out, B, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == held0


@pytest.mark.parametrize("kind", ["real", "mrecursion"])
def test_noalloc_refuses_real_and_order_recursion_plans(kind):
    from paper_2311_14670_gb300 import Plan
    from paper_2311_14670_gb300 import _native as nat

    L = 16
    plan = Plan(L, real=True) if kind == "real" else Plan(L, spin=1, mrecursion=True)
    x = torch.zeros(plan.coef_shape(1), dtype=plan.dtype, device="cuda")
    out = torch.zeros(plan.shape(1), dtype=plan.signal_dtype, device="cuda")
    with pytest.raises(nat.S2GBError) as e:
        nat.inverse_noalloc(plan._h, x, out, 1, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == nat.S2GB_EUNSUPPORTED


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    from paper_2311_14670_gb300 import Plan
    from paper_2311_14670_gb300 import _native as nat

    L, B = 1024, 4                      # 134 MB of theta-stage output alone
    plan = Plan(L, spin=0, max_batch=B)
    x = to_gpu(synth.flm_gaussian(L, 0, B, seed=1))
    out = torch.empty_like(x)
    with pytest.raises(nat.S2GBError) as e:
        nat.inverse_noalloc(plan._h, x, out, B, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == nat.S2GB_EWORKSPACE
