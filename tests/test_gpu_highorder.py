"""The high-order multigrid of the CUDA path (Sec. 4, the setting of p >= 4)
against the oracle's (oracle/highorder.py), through the C ABI.

The V-cycle: smoothing on the finest level by the subspace-corrected mass
smoother (fast diagonalization of a Kronecker sum of 1D pencils, rank-one
geometry approximation), L2-projection transfer to degree 1 on half the
elements and the standard V-cycle of that space, back, smoothing again.  It
is a linear operator; GPU and oracle apply the same one, so every output
entry is compared.  The two sides build the 1D pencils independently (GPU:
host FP64 Jacobi eigensolver; oracle: LAPACK), so their eigenvector bases
differ within clusters of close eigenvalues, but the operator
U diag(1/lambda) U^T does not.  Bars as for the standard V-cycle: FP64
max(1e-12, 4 eps64 max(kappa(A_0), kappa(A_fine))); FP32 (mixed path)
max(1e-5, 4 eps32 kappa(A_0)), A_0 the coarsest degree-1 operator, raised to
four times the V-cycle's sensitivity to the FP32 storage of the fine
operator where that is larger: the oracle's V-cycle applied once more with
its fine operator rounded to FP32 (what the mixed path stores) differs from
the FP64 one by 3.5e-4 on a degree-7 patch (eps32 times an effective
condition of about 3e3; rounding U, the scaling or P to FP32 moves it by
less than 1e-8), while an order-one mistake moves it by 1e-1 and more.

End to end: IETI-DP with the high-order V-cycle as the local solver's
preconditioner against the conforming global direct solve (relative error
<= 1e-8), outer iterations within +-1 of the oracle's run with the same
multigrid, and on the FP64 path the mean inner CG iteration count within +-1.
"""
import copy

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import ietidp as O
from oracle.domain import Multipatch
from paper_1705_04531_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp
    return ietidp


def _uneven():
    return W.Domain(2, (2, 2), [[5, 7], [7, 5]], [[8, 8], [8, 16]], W.UNIT, {"kind": "sin2d"},
                    (W.PRIMAL_VERTEX, W.PRIMAL_EDGE), "uneven_ho")


DOMS = {
    "square_p4_n16": lambda: W.random_quad_rhs(W.uniform_grid(2, (2, 2), 4, 16), seed=3),
    "annulus3x3_p5_floating": lambda: W.annulus_6x6(8, 5, grid=(3, 3)),
    "uneven_p5_p7": lambda: W.random_quad_rhs(_uneven(), seed=5),
    "cube_p4": lambda: W.random_quad_rhs(W.cube_2x2x2(4, 4), seed=7),
    # curved patches on which the high-order V-cycle overshoots (eigenvalues
    # of V K above 1): the primal basis must come from the standard hierarchy
    "annulus3x3_p4_n16": lambda: W.annulus_6x6(16, 4, grid=(3, 3)),
}

_ORC = {}


def _oracle(name):
    if name not in _ORC:
        _ORC[name] = O.IETIDP(DOMS[name](), O.Options(mode="mg", mg_kind="highorder"))
    return _ORC[name]


def _fp32_operator_sensitivity(mg, b, ref):
    """Relative change of the oracle's V-cycle when its fine operator is
    rounded to FP32."""
    m = copy.copy(mg)
    m.Af = mg.Af.astype(np.float32).astype(np.float64)
    return float(np.abs(m.vcycle(b.copy()) - ref).max() / np.abs(ref).max())


def _kappa(A):
    A = A.tocsc()
    if A.shape[0] <= 2000:
        return float(np.linalg.cond(A.toarray())) if A.shape[0] else 1.0
    lmax = spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = spla.eigsh(A, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    return float(lmax / lmin)


@pytest.mark.parametrize("hierarchy", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(DOMS))
def test_highorder_vcycle_matches_oracle(api, name, prec, hierarchy):
    orc = _oracle(name)
    dom = orc.dom
    prob = api.Problem(dom)
    sol = api.Solver(prob, precision=prec, mg_kind="highorder")
    rng = np.random.default_rng(21)
    b = torch.tensor(rng.standard_normal(sol.n_torn), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    sol.vcycles_hierarchy(hierarchy, b, x, 1)
    torch.cuda.synchronize()
    bs, xs = sol.split(b), sol.split(x)
    worst = 0.0
    for k in range(dom.npatch):
        mg = orc.mgN[k] if hierarchy == 0 else orc.mgD[k]
        fr = mg.free
        ref = mg.vcycle(bs[k][fr].copy())
        got = xs[k]
        mask = np.ones(len(got), dtype=bool)
        mask[fr] = False
        assert np.all(got[mask] == 0.0), "masked entries must stay untouched"
        scale = float(np.abs(ref).max())
        err = float(np.abs(got[fr] - ref).max()) / scale
        k0 = _kappa(mg.coarse.A[0])
        if prec == "fp64":
            bar = max(1e-12, 4.0 * EPS64 * max(k0, _kappa(mg.Af)))
        else:
            bar = max(1e-5, 4.0 * EPS32 * k0, 4.0 * _fp32_operator_sensitivity(mg, bs[k][fr], ref))
        worst = max(worst, err / bar)
        assert err <= bar, (k, err, bar)
    print(f"{name} {prec} hierarchy={hierarchy}: worst error / bar = {worst:.3f}")
    sol.close()
    prob.close()


def relerr(got, ref):
    return np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(got, ref)) / sum(np.sum(b ** 2) for b in ref))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", list(DOMS))
def test_highorder_solve_matches_global(api, name, prec):
    orc = _oracle(name)
    dom = orc.dom
    mp = Multipatch(dom)
    ref = mp.to_patches(mp.solve_global())
    prob = api.Problem(dom)
    sol = api.Solver(prob, precision=prec, mg_kind="highorder")
    u, st = sol.solve()
    err = relerr(sol.split(u), ref)
    assert st["converged"] and err <= 1e-8, (err, st)
    if orc.stats.outer_it == 0:
        orc.solve()
    assert abs(st["outer_it"] - orc.stats.outer_it) <= 1, (st["outer_it"], orc.stats.outer_it)
    its = [i for i in orc.stats.neumann_its if i > 0]
    print(f"{name} {prec}: outer {st['outer_it']} (oracle {orc.stats.outer_it}), inner mean "
          f"{st['inner_it_avg']:.2f} (oracle {np.mean(its):.2f})")
    if prec == "fp64":
        assert abs(st["inner_it_avg"] - np.mean(its)) <= 1.0, (st["inner_it_avg"], np.mean(its))
    sol.close()
    prob.close()
