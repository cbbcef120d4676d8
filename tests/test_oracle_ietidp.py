"""Pins of the IETI-DP oracle (Sec. 2-4): its solution equals the conforming
global direct solve in all three modes (D-D, D-MG, MG-MG), jumps vanish, the primal basis solves Eq. 6, MG-MG
equals D-D, the Lanczos condition estimate equals the spectrum of the
preconditioned dual operator, and kappa grows like (1 + log(H/h))^2."""
import numpy as np
import pytest

from oracle import ietidp
from oracle.domain import Multipatch
from paper_1705_04531_gb300 import workloads as W

CASES = [
    lambda: W.random_quad_rhs(W.square_2x2(8, 2)),
    lambda: W.annulus_6x6(8, 3, grid=(3, 3)),
    lambda: W.random_quad_rhs(W.cube_2x2x2(4, 2)),
    lambda: W.random_quad_rhs(W.uneven_8x8(0, grid=(3, 2), nelems=(4, 8))),
]


def _relerr(u, ref):
    return np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(u, ref))
                   / sum(np.sum(b ** 2) for b in ref))


@pytest.mark.parametrize("mode", ["direct", "mg", "dmg"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_equals_global_solve(case, mode):
    dom = CASES[case]()
    mp = Multipatch(dom)
    ref = mp.to_patches(mp.solve_global())
    s = ietidp.IETIDP(dom, ietidp.Options(mode=mode))
    u = s.solve()
    assert s.stats.converged and s.stats.outer_it > 0
    assert _relerr(u, ref) < 1e-10
    unorm = np.sqrt(sum(np.sum(x ** 2) for x in u))
    assert np.linalg.norm(s.jump(u)) < 1e-10 * unorm


@pytest.mark.parametrize("mode", ["direct", "mg"])
def test_primal_basis_eq6(mode):
    dom = W.annulus_6x6(8, 3, grid=(3, 3))
    s = ietidp.IETIDP(dom, ietidp.Options(mode=mode))
    rng = np.random.default_rng(0)
    for k in range(s.N):
        C, phi, K = s.C[k].toarray(), s.phi[k], s.K[k]
        assert np.abs(C @ phi - np.eye(C.shape[0])).max() < 1e-12
        v = rng.standard_normal(K.shape[0])
        v -= C.T @ np.linalg.solve(C @ C.T, C @ v)        # v in ker C
        assert np.abs(phi.T @ (K @ v)).max() < 1e-9 * np.linalg.norm(K @ v)


def test_mg_basis_equals_direct_basis():
    dom = W.annulus_6x6(8, 3, grid=(3, 3))
    a = ietidp.IETIDP(dom, ietidp.Options(mode="direct"))
    b = ietidp.IETIDP(dom, ietidp.Options(mode="mg"))
    for k in range(a.N):
        assert np.abs(a.phi[k] - b.phi[k]).max() < 1e-9
    assert np.abs(a.SPiPi - b.SPiPi).max() < 1e-9 * np.abs(a.SPiPi).max()


def test_edge_average_weights():
    """Edge rows of C are the normalized integrals of the tangential basis
    functions over the edge's interior dofs; vertex rows are unit rows."""
    dom = W.annulus_6x6(6, 2, grid=(2, 2))
    s = ietidp.IETIDP(dom, ietidp.Options(mode="direct"))
    t = np.concatenate([np.zeros(3), np.arange(1, 6) / 6, np.ones(3)])
    ints = np.array([(t[i + 3] - t[i]) / 3 for i in range(8)])[1:-1]
    w = ints / ints.sum()
    for k in range(s.N):
        for row in s.C[k].toarray():
            nz = row[row != 0]
            if len(nz) == 1:
                assert nz[0] == 1.0
            else:
                assert np.allclose(np.sort(nz), np.sort(w), atol=1e-15)


def _open_knot_integrals(n, p):
    """Integrals of the n+p B-splines of degree p on the open uniform knot
    vector of n elements over (0,1): (t_{i+p+1} - t_i) / (p + 1)."""
    t = np.concatenate([np.zeros(p + 1), np.arange(1, n) / n, np.ones(p + 1)])
    return np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(n + p)])


def test_face_average_weights():
    """3D face rows of C: the weight of the face function (j_a, j_b) is the
    product of the two tangential 1D basis integrals over the face's interior
    functions (the trace minus its edges), normalised to sum 1.  Every
    direction has its own degree and element count, so that a wrong
    tangential pair, a transposed pair or a missing normalisation changes the
    expected weight of some position."""
    degree = [[2, 2], [3, 3], [2]]
    nelem = [[4, 4], [5, 5], [6]]
    dom = W.Domain(3, (2, 2, 1), degree, nelem, W.UNIT, {"kind": "sin3d"},
                   (W.PRIMAL_VERTEX, W.PRIMAL_EDGE, W.PRIMAL_FACE), "face_pin")
    dom = W.random_quad_rhs(dom, seed=7)
    s = ietidp.IETIDP(dom, ietidp.Options(mode="direct"))
    m = [nelem[r][0] + degree[r][0] for r in range(3)]
    ints = [_open_knot_integrals(nelem[r][0], degree[r][0]) for r in range(3)]
    nface = 0
    for k in range(s.N):
        fr = s.free[k]
        for row in s.C[k].toarray():
            nzl = np.nonzero(row)[0]
            if len(nzl) <= 1:
                continue
            full = fr[nzl]
            ti = [full % m[0], (full // m[0]) % m[1], full // (m[0] * m[1])]
            const = [r for r in range(3) if np.all(ti[r] == ti[r][0])]
            if len(const) != 1:
                continue                      # an edge row (two fixed directions)
            nface += 1
            normal = const[0]
            assert ti[normal][0] in (0, m[normal] - 1)
            tang = [r for r in range(3) if r != normal]
            # the interior functions of the face, all of them present
            for r in tang:
                assert set(ti[r]) == set(range(1, m[r] - 1))
            w = ints[tang[0]][ti[tang[0]]] * ints[tang[1]][ti[tang[1]]]
            den = ints[tang[0]][1:-1].sum() * ints[tang[1]][1:-1].sum()
            assert np.allclose(row[nzl], w / den, rtol=1e-14, atol=0)
    # 2x2x1 grid: four interior faces, each seen from both of its patches
    assert nface == 8


def test_lanczos_kappa_matches_spectrum():
    dom = W.random_quad_rhs(W.square_2x2(8, 2))
    s = ietidp.IETIDP(dom, ietidp.Options(mode="direct", tol_outer=1e-14))
    s.solve()
    n = s.nlam
    F = np.array([s.F(e) for e in np.eye(n)]).T
    M = np.array([s.precond(e) for e in np.eye(n)]).T
    ev = np.sort(np.linalg.eigvals(M @ F).real)
    ev = ev[ev > 1e-8 * ev[-1]]
    kap = ev[-1] / ev[0]
    assert abs(s.stats.kappa - kap) < 1e-6 * kap


def test_kappa_log_growth():
    """kappa / (1 + log(H/h))^2 must not grow under refinement (Sec. 4:
    the logarithmic dependence of the condition number on h)."""
    ratios = []
    kappas = []
    for n in (4, 8, 16, 32):
        dom = W.annulus_6x6(n, 2, grid=(3, 3))
        s = ietidp.IETIDP(dom, ietidp.Options(mode="direct"))
        s.solve()
        kappas.append(s.stats.kappa)
        ratios.append(s.stats.kappa / (1 + np.log(n)) ** 2)
    assert all(np.diff(kappas) > -1e-6)
    assert ratios[-1] <= ratios[0] + 1e-9


def test_symmetric_problem_has_zero_dual_rhs():
    dom = W.square_2x2(8, 2)           # f symmetric under both mirrors
    s = ietidp.IETIDP(dom, ietidp.Options(mode="direct"))
    u = s.solve()
    assert s.stats.outer_it == 0 and s.stats.d_norm < 1e-12 * s.stats.d_scale
    mp = Multipatch(dom)
    assert _relerr(u, mp.to_patches(mp.solve_global())) < 1e-12


def test_single_patch_has_no_multipliers():
    dom = W.uniform_grid(2, (1, 1), 3, 8)
    s = ietidp.IETIDP(dom, ietidp.Options(mode="mg"))
    u = s.solve()
    assert s.nlam == 0 and s.nPi == 0
    mp = Multipatch(dom)
    assert _relerr(u, mp.to_patches(mp.solve_global())) < 1e-11


@pytest.mark.parametrize("case", range(len(CASES)))
def test_dmg_iterations_equal_mgmg(case):
    """D-MG and MG-MG share the preconditioner (Dirichlet problems by
    multigrid); their Neumann solves differ only by the inner tolerance, so
    the outer iteration counts agree to within one."""
    dom = CASES[case]()
    a = ietidp.IETIDP(dom, ietidp.Options(mode="dmg"))
    a.solve()
    b = ietidp.IETIDP(dom, ietidp.Options(mode="mg"))
    b.solve()
    assert abs(a.stats.outer_it - b.stats.outer_it) <= 1


def test_no_primal_dofs_on_a_strip():
    """Degenerate case: a 3x1 strip with vertex primal constraints only has
    every cross point on the Dirichlet boundary, so n_Pi = 0 and no patch
    floats; K~ is then block diagonal and the method is plain tearing and
    interconnecting.  The solution still equals the global direct solve."""
    dom = W.random_quad_rhs(W.uniform_grid(2, (3, 1), 2, 8, W.UNIT, None, ("vertex",)), seed=9)
    mp = Multipatch(dom)
    ref = mp.to_patches(mp.solve_global())
    for mode in ("direct", "mg"):
        s = ietidp.IETIDP(dom, ietidp.Options(mode=mode))
        u = s.solve()
        assert s.nPi == 0 and not any(s.floating) and s.nlam > 0
        assert s.stats.converged and _relerr(u, ref) < 1e-10
