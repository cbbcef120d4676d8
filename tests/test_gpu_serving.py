"""Continuous-batching server (the serving pattern): requests of
different sizes, admitted by device-memory budget, overlap on the GPU; each
result is the same alone and in the mix, and matches the oracle's direct
solve."""
import numpy as np
import pytest

from oracle.domain import Multipatch
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


def _requests(n=6, seed=7):
    reqs = W.serving_stream(nreq=n, rate=1000.0, seed=seed, ms=(2, 3, 4), ps=(2, 3), ns=(8, 16))
    return [r.domain for r in reqs]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_alone_equals_mix(api, prec):
    doms = _requests()
    srv = api.Server(8 << 30, max_concurrent=4, precision=prec)
    alone = []
    for d in doms:
        t = srv.submit(d)
        state, u, st, tm = srv.wait(t)
        assert st["converged"]
        alone.append(u)
    tickets = [srv.submit(d) for d in doms]
    mixed = [srv.wait(t)[1] for t in tickets]
    srv.close()
    for a, b in zip(alone, mixed):
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())
    # and against the definition: conforming global direct solve
    for d, u in zip(doms[:3], alone[:3]):
        mp = Multipatch(d)
        ref = np.concatenate(mp.to_patches(mp.solve_global()))
        assert np.linalg.norm(u - ref) <= 1e-8 * np.linalg.norm(ref)


def test_budget_admission(api):
    doms = _requests(4, seed=3)
    est = None
    srv = api.Server(1 << 40, max_concurrent=2)
    est = max(srv.estimate(d) for d in doms)
    srv.close()
    # a budget that fits exactly one request at a time still serves them all
    srv = api.Server(est, max_concurrent=4)
    tickets = [srv.submit(d) for d in doms]
    peak = 0
    while True:
        s = srv.status()
        peak = max(peak, s["running"])
        if s["running"] == 0 and s["queued"] == 0:
            break
    outs = [srv.wait(t) for t in tickets]
    srv.close()
    assert all(o[0] == 2 and o[2]["converged"] for o in outs)
    # over-budget requests are rejected at submission
    srv = api.Server(1 << 20, max_concurrent=1)
    with pytest.raises(api.IetidpError):
        srv.submit(doms[0])
    srv.close()
