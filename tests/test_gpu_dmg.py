"""D-MG on the GPU (method IETIDP_METHOD_DMG, Sec. 3.3): direct local Neumann
solves by banded Cholesky (pinned dof on floating patches), multigrid
Dirichlet problems, through the C ABI against the CPU oracle's D-MG mode.

Bars: relative solution error <= 1e-8 against the conforming direct solve
(FP64 and mixed V-cycles in the preconditioner); outer iterations within +-1
of the oracle's D-MG; batched = single; the factorization guard rejects a
band too large to factor; the substitution vector in global memory (patches
above the shared-memory cap) gives the same bits as in shared memory; bands
wider than a CTA's threads (3D patches) take the strided sweep; the server
with method D-MG gives each request the same result alone and in the mix."""
import os

import numpy as np
import pytest

from oracle import assembly
from oracle import ietidp as O
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
    "square_rq": lambda: W.random_quad_rhs(W.square_2x2(16, 2), seed=41),
    "annulus3x3": lambda: W.annulus_6x6(8, 3, grid=(3, 3)),
    "uneven3x3": lambda: W.random_quad_rhs(W.uneven_8x8(0, grid=(3, 3), nelems=(8, 16, 32)), seed=42),
    "modes4x4": lambda: W.uniform_grid(2, (4, 4), 3, 16, W.UNIT,
                                       W.sine_modes_rhs(np.random.default_rng(43)), ("vertex", "edge")),
    "cube_rq": lambda: W.random_quad_rhs(W.cube_2x2x2(8, 2), seed=44),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(DOMS))
def test_dmg_matches_direct_and_oracle(api, name, prec):
    dom = DOMS[name]()
    mp = Multipatch(dom)
    ref = mp.to_patches(mp.solve_global())
    sol = api.Solver(api.Problem(dom), precision=prec, method="dmg")
    u, st = sol.solve()
    err = relerr(sol.split(u), ref)
    assert st["converged"] and err <= 1e-8, (err, st)
    orc = O.IETIDP(dom, O.Options(mode="dmg"))
    orc.solve()
    assert abs(st["outer_it"] - orc.stats.outer_it) <= 1, (st["outer_it"], orc.stats.outer_it)


def test_dmg_batch_equals_single(api):
    doms = [DOMS[n]() for n in ("square_rq", "annulus3x3", "uneven3x3")]
    sols = [api.Solver(api.Problem(d), precision="mixed", method="dmg") for d in doms]
    singles = [s.solve()[0].clone() for s in sols]
    us, sts = api.Solver.solve_batch(sols)
    for s, a, b, st in zip(sols, singles, us, sts):
        assert st["converged"]
        assert relerr(s.split(b), s.split(a)) <= 1e-10


def test_dmg_rejects_oversized_band(api):
    # 2x2x2 cube, p=2, 32^3 elements per patch: band 2382, n 39304 -> n bw^2 ~ 2.2e11
    prob = api.Problem(W.cube_2x2x2(32, 2))
    with pytest.raises(api.IetidpError) as e:
        api.Solver(prob, method="dmg")
    assert api.ERRORS[e.value.code] == "INVALID_ARG"


def test_dmg_global_vector_path_equals_shared(api):
    dom = DOMS["annulus3x3"]()
    prob = api.Problem(dom)
    u1, st1 = api.Solver(prob, precision="mixed", method="dmg").solve()
    u1 = u1.clone()
    os.environ["IETIDP_DIRECT_SMEM"] = "0"
    try:
        u0, st0 = api.Solver(prob, precision="mixed", method="dmg").solve()
    finally:
        del os.environ["IETIDP_DIRECT_SMEM"]
    assert torch.equal(u0, u1)
    assert st0["outer_it"] == st1["outer_it"]


def test_dmg_wide_band_3d(api):
    """2x2x2 cube, p=2, 16^3 elements per patch: 18^3 = 5832 functions and a
    band of 2 + 18 (2 + 18 * 2) = 686 offsets, more than the 512 threads of a
    solve.  Checked by continuity of the torn copies and by sampled interior
    rows of the conforming system computed one by one by the oracle."""
    dom = W.random_quad_rhs(W.cube_2x2x2(16, 2), seed=45)
    sol = api.Solver(api.Problem(dom), precision="mixed", method="dmg")
    u, st = sol.solve()
    assert st["converged"]
    got = sol.split(u)
    mp = Multipatch(dom)
    hi = np.full(mp.nglob, -np.inf)
    lo = np.full(mp.nglob, np.inf)
    for k, uk in enumerate(got):
        np.maximum.at(hi, mp.l2g[k], uk)
        np.minimum.at(lo, mp.l2g[k], uk)
    assert np.max(hi - lo) <= 1e-9 * np.max(np.abs(hi))
    rng = np.random.default_rng(1)
    m = 18
    for k in (0, 3, 7):
        for _ in range(4):
            i0, i1, i2 = (int(rng.integers(1, m - 1)) for _ in range(3))
            i = i0 + m * (i1 + m * i2)
            cols, vals, fi = assembly.row_stiffness_load(dom, k, i)
            ku = float(vals @ got[k][cols])
            scale = float(np.abs(vals) @ np.abs(got[k][cols])) + abs(fi)
            assert abs(ku - fi) <= 1e-9 * scale, (k, i, ku, fi)


def test_dmg_server_alone_equals_mix(api):
    """Serving with method D-MG: each request's result is the same alone and
    in the mix (continuous batching) and equals the direct solve."""
    reqs = [r.domain for r in W.serving_stream(nreq=4, rate=1000.0, seed=46, ms=(2, 3), ps=(2, 3), ns=(8, 16))]
    srv = api.Server(8 << 30, max_concurrent=2, precision="mixed", method="dmg")
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
