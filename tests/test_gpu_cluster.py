"""Local solves on thread-block clusters: one slot's rows split over 2, 4 or 8
CTAs (Eq. 7 Neumann solves, the Dirichlet solves of the scaled Dirichlet
preconditioner and the V-cycles, Sec. 3-4), vectors in global memory,
cluster barriers between color steps, dot products summed over the cluster
in rank order.

The split changes nothing in the arithmetic of a row, only the order of the
partial sums of the dot products (per CTA, then over the CTAs), so a solve
on clusters agrees with the one-CTA-per-slot solve to the rounding of those
sums amplified by the CG (bar 1e-10 relative, the batch-versus-single bar of
the engine tests; 1e-9 on the mixed path, whose one-CTA solve applies the
CG's operator in FP32 pairs) and with the conforming direct solve to 1e-8, with the
same outer iteration count (+-1).  IETIDP_CLUSTERS forces the cluster size
on every group that can take it.
"""
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


DOMS = {
    "annulus3x3_floating": lambda: W.random_quad_rhs(W.annulus_6x6(16, 3, grid=(3, 3)), seed=2),
    "uneven3x3": lambda: W.random_quad_rhs(W.uneven_8x8(0, grid=(3, 3), nelems=(8, 16, 32)), seed=4),
    "cube_3d": lambda: W.random_quad_rhs(W.cube_2x2x2(8, 2), seed=6),
}


def _solve(api, dom, prec, clusters, monkeypatch):
    monkeypatch.setenv("IETIDP_CLUSTERS", str(clusters))
    prob = api.Problem(dom)
    sol = api.Solver(prob, precision=prec)
    u, st = sol.solve()
    torch.cuda.synchronize()
    got = sol.split(u)
    sol.close()
    prob.close()
    monkeypatch.delenv("IETIDP_CLUSTERS", raising=False)
    return got, st


@pytest.mark.parametrize("csize", [2, 4, 8])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(DOMS))
def test_cluster_solve_matches_single_cta(api, name, prec, csize, monkeypatch):
    dom = DOMS[name]()
    ref = Multipatch(dom)
    uref = ref.to_patches(ref.solve_global())
    u1, st1 = _solve(api, dom, prec, 0, monkeypatch)
    uc, stc = _solve(api, dom, prec, csize, monkeypatch)
    assert stc["converged"], stc
    assert relerr(uc, uref) <= 1e-8, relerr(uc, uref)
    # mixed: the one-CTA solve applies the CG's operator in FP32 pairs, the
    # cluster (global-vector variant) in FP64; both to the outer tolerance
    assert relerr(uc, u1) <= (1e-10 if prec == "fp64" else 1e-9), relerr(uc, u1)
    assert abs(stc["outer_it"] - st1["outer_it"]) <= 1, (stc["outer_it"], st1["outer_it"])
    tab = api.autotune_table()
    assert all("cluster" in t for t in tab)


def test_cluster_vcycles_match_single_cta(api, monkeypatch):
    dom = W.annulus_6x6(16, 3, grid=(3, 3))
    outs = []
    for cl in (0, 4):
        monkeypatch.setenv("IETIDP_CLUSTERS", str(cl))
        prob = api.Problem(dom)
        sol = api.Solver(prob, precision="fp64")
        f = prob.load()
        x = torch.zeros_like(f)
        api.Solver.vcycles_batch([sol], [f], [x], 2)
        torch.cuda.synchronize()
        outs.append(x.cpu().numpy())
        sol.close()
        prob.close()
    monkeypatch.delenv("IETIDP_CLUSTERS", raising=False)
    scale = np.abs(outs[0]).max()
    # the same operator; only the coarse levels' row sums are split over
    # lane groups in a different pattern (rounding order)
    assert np.abs(outs[1] - outs[0]).max() <= 1e-10 * scale
