"""The allocation-free V-cycle entry point against the regular one.

ietidp_vcycles_noalloc serves callers that cannot allocate device memory
when they run the smoother: a plugin inside a host framework that owns the
device memory pool and forbids allocations outside it, or a latency-bound
loop that must not call cudaMalloc/cudaFree, which may synchronize the
device and take unbounded time.  Its scratch is a static device array
instead of the handle's buffers, so its output must match ietidp_vcycles,
call after call, including after another handle has used the array, and on
a domain whose slots run on several kernel specialisations at once.  A warm
call must leave the device's free memory unchanged, and a problem whose
scratch exceeds the array is rejected.  Collected last so that a run
stopping at the first failure has run every other test first."""
import numpy as np
import pytest

from paper_1705_04531_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp
    return ietidp


def _reference(sol, ncycles, seed=0):
    g = torch.Generator(device="cuda").manual_seed(seed)
    e = torch.rand(sol.n_torn, dtype=torch.float64, device="cuda", generator=g)
    b = torch.empty_like(e)
    sol.apply_K(e, b)
    ref = torch.zeros_like(b)
    sol.vcycles(b, ref, ncycles)
    torch.cuda.synchronize()
    return b, ref


def _check_calls(sol, b, ref, ncycles, calls=2):
    scale = float(ref.abs().max())
    assert scale > 0
    for _ in range(calls):                  # calls in a row share the static scratch
        got = torch.zeros_like(b)
        sol.vcycles_noalloc(b, got, ncycles)
        torch.cuda.synchronize()
        assert float((got - ref).abs().max()) <= 1e-12 * scale


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_vcycles_match(api, prec):
    dom = W.annulus_6x6(16, 3, grid=(3, 3))
    prob = api.Problem(dom)
    sol = api.Solver(prob, precision=prec)
    b, ref = _reference(sol, 2)
    _check_calls(sol, b, ref, 2)
    sol.close()
    prob.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_after_other_handle_and_several_specialisations(api, prec):
    """Another handle writes the shared array first; the uneven-degree domain
    then runs its specialisation groups concurrently on side streams, each
    slot in its own part of the array."""
    other = api.Solver(api.Problem(W.annulus_6x6(8, 3, grid=(3, 3))), precision=prec)
    bo, _ = _reference(other, 1, seed=3)
    xo = torch.zeros_like(bo)
    other.vcycles_noalloc(bo, xo, 1)
    dom = W.uneven_8x8(0, grid=(3, 3), nelems=(8, 16, 32))
    prob = api.Problem(dom)
    sol = api.Solver(prob, precision=prec)
    b, ref = _reference(sol, 2, seed=1)
    _check_calls(sol, b, ref, 2)
    other.close()
    sol.close()
    prob.close()


def test_noalloc_warm_call_keeps_free_memory(api):
    prob = api.Problem(W.annulus_6x6(16, 3, grid=(3, 3)))
    sol = api.Solver(prob, precision="mixed")
    b, ref = _reference(sol, 1)
    x = torch.zeros_like(b)
    sol.vcycles_noalloc(b, x, 1)              # warm: kernels and streams in use
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        x.zero_()
        sol.vcycles_noalloc(b, x, 1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    sol.close()
    prob.close()


def test_noalloc_rejects_problem_above_limit(api):
    """6x6 annulus with 128 x 128 elements per patch: its FP64 scratch alone
    (36 patches x 5 vectors x 131^2 doubles, about 25 MB) exceeds the 16 MiB
    array, so the call is refused before any device work."""
    prob = api.Problem(W.annulus_6x6(128, 3))
    sol = api.Solver(prob, precision="mixed")
    b = torch.ones(sol.n_torn, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(api.IetidpError) as ei:
        sol.vcycles_noalloc(b, x, 1)
    assert ei.value.code == -1 and "static limit" in str(ei.value)
    assert float(x.abs().max()) == 0.0
    sol.close()
    prob.close()
