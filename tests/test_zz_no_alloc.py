"""The allocation-free V-cycle entry point against the regular one.

ietidp_vcycles_noalloc serves callers that cannot allocate device memory
when they run the smoother (a plugin inside a framework that owns the device
memory pool, or a latency-bound loop that must not call cudaMalloc/cudaFree).
Its scratch is a static device array instead of the handle's buffers, so its
output must match ietidp_vcycles, call after call.  Collected last so that a
run stopping at the first failure has run every other test first."""
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_vcycles_match(api, prec):
    dom = W.annulus_6x6(16, 3, grid=(3, 3))
    prob = api.Problem(dom)
    sol = api.Solver(prob, precision=prec)
    e = torch.rand(sol.n_torn, dtype=torch.float64, device="cuda")
    b = torch.empty_like(e)
    sol.apply_K(e, b)
    ref = torch.zeros_like(b)
    sol.vcycles(b, ref, 2)
    torch.cuda.synchronize()
    scale = float(ref.abs().max())
    assert scale > 0
    for _ in range(2):                      # two calls in a row share the static scratch
        got = torch.zeros_like(b)
        sol.vcycles_noalloc(b, got, 2)
        torch.cuda.synchronize()
        assert float((got - ref).abs().max()) <= 1e-12 * scale
    sol.close()
    prob.close()
