"""MG-MG-S on the GPU (method IETIDP_METHOD_SADDLE): Bramble-Pasciak CG on the
saddle-point system of Eq. 2 through the C ABI, against the CPU oracle.

Bars: relative solution error <= 1e-8 against the conforming direct solve
(FP64 and mixed V-cycles); BPCG iteration counts within +-1 of the oracle's
MG-MG-S on the FP64 path; the mixed path restarts from an FP64 residual after
every 1e-4 of reduction (refinement against the FP32 rounding of its
V-cycles: two restarts at tolerance 1e-10) and may take one iteration fewer
or up to one more per restart, plus one; batched and served results equal
the single solves to rounding.
"""
import numpy as np
import pytest

from oracle import ietidp as O
from oracle import saddle
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


DOMS = {
    "square_rq": lambda: W.random_quad_rhs(W.square_2x2(16, 2), seed=31),
    "annulus3x3": lambda: W.annulus_6x6(8, 3, grid=(3, 3)),
    "uneven3x3": lambda: W.random_quad_rhs(W.uneven_8x8(0, grid=(3, 3), nelems=(8, 16, 32)), seed=32),
    "modes4x4": lambda: W.uniform_grid(2, (4, 4), 3, 16, W.UNIT,
                                       W.sine_modes_rhs(np.random.default_rng(33)), ("vertex", "edge")),
    "cube_rq": lambda: W.random_quad_rhs(W.cube_2x2x2(8, 2), seed=34),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(DOMS))
def test_saddle_matches_direct_and_oracle(api, name, prec):
    dom = DOMS[name]()
    mp = Multipatch(dom)
    ref = mp.to_patches(mp.solve_global())
    sol = api.Solver(api.Problem(dom), precision=prec, method="saddle")
    u, st = sol.solve()
    got = sol.split(u)
    err = relerr(got, ref)
    assert st["converged"] and err <= 1e-8, (err, st)
    orc = O.IETIDP(dom, O.Options(mode="mg"))
    _, ost = saddle.bpcg(orc)
    if prec == "fp64":
        assert abs(st["outer_it"] - ost["iterations"]) <= 1, (st["outer_it"], ost["iterations"])
    else:
        # FP32 V-cycles: the residual is recomputed in FP64 after every 1e-4
        # of reduction (two restarts at tolerance 1e-10); each restart drops
        # the recursion's history and may cost one iteration
        restarts = 2
        print(name, "mixed BPCG", st["outer_it"], "oracle FP64", ost["iterations"])
        assert ost["iterations"] - 1 <= st["outer_it"] <= ost["iterations"] + 1 + restarts, (
            st["outer_it"], ost["iterations"])
    assert st["vcycles"] > 0


def test_saddle_batch_equals_single(api):
    doms = [DOMS[n]() for n in ("square_rq", "annulus3x3", "uneven3x3")]
    sols = [api.Solver(api.Problem(d), precision="mixed", method="saddle") for d in doms]
    singles = [s.solve()[0].clone() for s in sols]
    us, sts = api.Solver.solve_batch(sols)
    for s, a, b, st in zip(sols, singles, us, sts):
        assert st["converged"]
        assert relerr(s.split(b), s.split(a)) <= 1e-10


def test_batch_rejects_mixed_methods(api):
    d = DOMS["square_rq"]()
    s1 = api.Solver(api.Problem(d), method="saddle")
    s2 = api.Solver(api.Problem(d), method="dual")
    with pytest.raises(api.IetidpError):
        api.Solver.solve_batch([s1, s2])


def test_saddle_server_alone_equals_mix(api):
    reqs = [r.domain for r in W.serving_stream(nreq=4, rate=1000.0, seed=35, ms=(2, 3), ps=(2, 3), ns=(8, 16))]
    srv = api.Server(8 << 30, max_concurrent=2, precision="mixed", method="saddle")
    alone = []
    for d in reqs:
        state, u, st, tm = srv.wait(srv.submit(d))
        assert st["converged"]
        alone.append(u)
    mixed = [srv.wait(t)[1] for t in [srv.submit(d) for d in reqs]]
    srv.close()
    for d, a, b in zip(reqs, alone, mixed):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)
        mp = Multipatch(d)
        ref = np.concatenate(mp.to_patches(mp.solve_global()))
        assert np.linalg.norm(a - ref) <= 1e-8 * np.linalg.norm(ref)
