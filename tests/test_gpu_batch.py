"""Batched lockstep solves (ietidp_solve_batch) through the C ABI.

Every handle of a batch must give the conforming direct solution of its own
problem (relative error <= 1e-8, as single solves) and agree with its own
single solve to rounding (the merged launches may use another block size, so
the reduction order of dot products may differ; 1e-10 relative).  Problems of
different sizes, degrees and precisions share launches and leave the batch at
different iterations.
"""
import os

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


def relerr(got, ref):
    return np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(got, ref)) / sum(np.sum(b ** 2) for b in ref))


def _doms():
    return [
        W.random_quad_rhs(W.square_2x2(16, 2), seed=11),
        W.annulus_6x6(8, 3, grid=(3, 3)),
        W.random_quad_rhs(W.uneven_8x8(0, grid=(3, 3), nelems=(8, 16, 32)), seed=12),
        W.uniform_grid(2, (4, 4), 3, 16, W.UNIT, W.sine_modes_rhs(np.random.default_rng(13)), ("vertex", "edge")),
        W.random_quad_rhs(W.cube_2x2x2(8, 2), seed=14),
    ]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_direct_and_single(api, prec):
    doms = _doms()
    probs = [api.Problem(d) for d in doms]
    sols = [api.Solver(p, precision=prec) for p in probs]
    us, sts = api.Solver.solve_batch(sols)
    assert len(sts) == len(doms)
    its = []
    for d, s, u, st in zip(doms, sols, us, sts):
        mp = Multipatch(d)
        ref = mp.to_patches(mp.solve_global())
        got = s.split(u)
        err = relerr(got, ref)
        assert st["converged"] and err <= 1e-8, (d.name, err, st)
        u1, st1 = s.solve()
        assert relerr(got, s.split(u1)) <= 1e-10
        assert abs(st1["outer_it"] - st["outer_it"]) <= 1
        its.append(st["outer_it"])
    # the jobs leave the batch at different iterations
    assert len(set(its)) > 1


def test_batch_host_equals_device(api):
    doms = _doms()[:3]
    sols = [api.Solver(api.Problem(d), precision="mixed") for d in doms]
    fs = [s.problem.load() for s in sols]
    us, _ = api.Solver.solve_batch(sols, fs)
    uh, sts = api.Solver.solve_batch_host(sols, [f.cpu().numpy() for f in fs])
    for a, b, st in zip(us, uh, sts):
        assert st["converged"]
        assert np.array_equal(a.cpu().numpy(), b)


def test_batch_of_copies_equal_each_other(api):
    """Identical problems in one batch take identical arithmetic."""
    dom = W.annulus_6x6(8, 3, grid=(3, 3))
    sols = [api.Solver(api.Problem(dom), precision="mixed") for _ in range(4)]
    us, sts = api.Solver.solve_batch(sols)
    for u, st in zip(us[1:], sts[1:]):
        assert torch.equal(u, us[0])
        assert st["outer_it"] == sts[0]["outer_it"]


def test_batch_rejects_duplicate_handle(api):
    sol = api.Solver(api.Problem(W.square_2x2(16, 2)))
    with pytest.raises(api.IetidpError) as e:
        api.Solver.solve_batch([sol, sol])
    assert api.ERRORS[e.value.code] == "INVALID_ARG"


def test_autotune_records_and_can_be_disabled(api):
    dom = W.annulus_6x6(8, 3, grid=(3, 3))
    sols = [api.Solver(api.Problem(dom), precision="mixed") for _ in range(2)]
    api.Solver.solve_batch(sols)
    tab = api.autotune_table()
    assert tab and all(t["threads"] in (128, 256, 512) and t["ctas_per_sm"] >= 1 for t in tab)
    os.environ["IETIDP_AUTOTUNE"] = "0"
    try:
        us0, st0 = api.Solver.solve_batch(sols)
    finally:
        del os.environ["IETIDP_AUTOTUNE"]
    us1, st1 = api.Solver.solve_batch(sols)
    for a, b in zip(us0, us1):
        assert relerr([a.cpu().numpy()], [b.cpu().numpy()]) <= 1e-10


@pytest.mark.parametrize("method", ["dual", "saddle", "dmg"])
def test_zero_load_gives_zero_solution(api, method):
    """Degenerate input: f = 0 gives u = 0 at once (zero dual right-hand side,
    or zero first BPCG inner product), in every method."""
    dom = W.annulus_6x6(8, 3, grid=(3, 3))
    sol = api.Solver(api.Problem(dom), precision="mixed", method=method)
    f = torch.zeros(sol.n_torn, dtype=torch.float64, device="cuda")
    u, st = sol.solve(f)
    assert st["converged"]
    assert float(u.abs().max()) == 0.0
    assert st["outer_it"] == 0


@pytest.mark.parametrize("method", ["dual", "saddle", "dmg"])
def test_graph_replay_equals_eager(api, method):
    """The CUDA-graph replay of the per-iteration launches gives the same bits
    as eager launches (MG-MG, MG-MG-S and D-MG ticks)."""
    dom = W.annulus_6x6(8, 3, grid=(3, 3))
    sol = api.Solver(api.Problem(dom), precision="mixed", method=method)
    u1, st1 = sol.solve()
    u1 = u1.clone()
    os.environ["IETIDP_GRAPHS"] = "0"
    try:
        u0, st0 = sol.solve()
    finally:
        del os.environ["IETIDP_GRAPHS"]
    assert torch.equal(u0, u1)
    assert st0["outer_it"] == st1["outer_it"]
