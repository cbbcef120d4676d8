"""Pins of the high-order multigrid oracle (oracle/highorder.py; Sec. 4, the
setting of p >= 4: degree 1 below the finest level, L2-projection transfers,
subspace-corrected mass smoother with a rank-one geometry approximation)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assembly, highorder as H, splines
from oracle.domain import Multipatch
from oracle import ietidp as O
from paper_1705_04531_gb300 import workloads as W


def _spline_eval(n, p, coef, x):
    return splines.basis_funs(splines.open_uniform_knots(n, p), p, x) @ coef


def _fd_deriv(n, p, coef, x0, k):
    """k-th derivative at x0 from the spline's own values: on the end element
    the spline is a polynomial of degree p, fitted through p + 1 interior
    points and differentiated (independent of the oracle's derivative
    functionals)."""
    a = x0 if x0 == 0.0 else 1.0 - 1.0 / n
    xs = a + np.linspace(0.1, 0.9, p + 1) / n
    vals = _spline_eval(n, p, coef, xs)
    poly = np.polynomial.Polynomial.fit(xs, vals, p, domain=[a, a + 1.0 / n])
    return poly.deriv(k)(x0)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 7])
@pytest.mark.parametrize("lo,hi", [(False, False), (True, False), (True, True)])
def test_subspace_end_derivatives_and_inverse_inequality(p, lo, hi):
    n = 8
    C, free = H.split_1d(n, p, lo, hi)
    Z = sla.null_space(C)
    m = n + p
    for col in Z.T:
        coef = np.zeros(m)
        coef[free] = col
        scale = np.abs(coef).max()
        for end, dirichlet in ((0.0, lo), (1.0, hi)):
            if dirichlet:
                assert abs(_spline_eval(n, p, coef, np.array([end]))[0]) <= 1e-10 * scale
            for k in range(1, p):
                if (k % 2 == 0) == dirichlet:
                    assert abs(_fd_deriv(n, p, coef, end, k)) <= 1e-6 * scale * n ** k
    M = splines.mass_1d(n, p)[np.ix_(free, free)]
    K = splines.stiffness_1d(n, p)[np.ix_(free, free)]
    h = 1.0 / n
    lam_sub = sla.eigh(Z.T @ K @ Z, Z.T @ M @ Z, eigvals_only=True).max()
    assert lam_sub <= 12.0 / h ** 2 * (1 + 1e-10), (lam_sub * h * h)
    if p >= 4:
        # the outlier functions near the ends break it on the full space
        assert sla.eigh(K, M, eigvals_only=True).max() > 12.0 / h ** 2


def test_khat_blocks():
    n, p, sigma = 8, 5, 12.0
    C, free = H.split_1d(n, p, True, False)
    M = splines.mass_1d(n, p)
    K = splines.stiffness_1d(n, p)
    Kh, Mf = H.khat_1d(n, p, free, C, M, K, sigma)
    Z = sla.null_space(C)
    Mr = M[np.ix_(free, free)]
    Kr = K[np.ix_(free, free)]
    G = np.linalg.solve(Mr, C.T)                     # M-orthogonal complement of ker C
    rng = np.random.default_rng(0)
    u, v = Z @ rng.standard_normal(Z.shape[1]), G @ rng.standard_normal(G.shape[1])
    assert np.isclose(u @ Kh @ u, sigma * n * n * (u @ Mr @ u), rtol=1e-10)
    assert np.isclose(v @ Kh @ v, v @ Kr @ v, rtol=1e-10)
    assert abs(u @ Kh @ v) <= 1e-10 * np.sqrt((u @ Kh @ u) * (v @ Kh @ v))


def test_transfer_reproduces_linear_functions():
    """A linear function lies in both spaces; its degree-1 coefficients (values
    at the knots) map to its degree-p coefficients (values at the Greville
    abscissae)."""
    n, p = 8, 5
    P = H.l2_transfer_1d(n, p, n // 2, False, False)
    tc = splines.open_uniform_knots(n // 2, 1)
    tf = splines.open_uniform_knots(n, p)
    grev_c = np.array([tc[i + 1] for i in range(n // 2 + 1)])
    grev_f = np.array([tf[i + 1:i + p + 1].mean() for i in range(n + p)])
    g = lambda x: 0.3 + 2.0 * x
    assert np.allclose(P @ g(grev_c), g(grev_f), atol=1e-12)


def test_transfer_with_dirichlet_end():
    n, p = 8, 4
    P = H.l2_transfer_1d(n, p, n // 2, True, False)
    tc = splines.open_uniform_knots(n // 2, 1)
    tf = splines.open_uniform_knots(n, p)
    grev_c = np.array([tc[i + 1] for i in range(n // 2 + 1)])[1:]
    grev_f = np.array([tf[i + 1:i + p + 1].mean() for i in range(n + p)])[1:]
    assert np.allclose(P @ (1.7 * grev_c), 1.7 * grev_f, atol=1e-12)


def test_rank_one_weights():
    dom = W.annulus_6x6(8, 3, grid=(3, 3))
    k = 4
    om = H.rank_one_weights(dom, k)
    x = np.linspace(0.05, 0.95, 7)
    from oracle import geometry

    def A(xi):
        _, J = geometry.patch_map(dom, k, xi)
        Ji = np.linalg.inv(J)
        return np.einsum("qac,qbc->qab", Ji, Ji) * np.abs(np.linalg.det(J))[:, None, None]
    for r in range(2):
        # exact on the two lines through the centre
        for s in range(2):
            xi = np.full((len(x), 2), 0.5)
            xi[:, s] = x
            approx = om[r][0](xi[:, 0]) * om[r][1](xi[:, 1])
            assert np.allclose(approx, A(xi)[:, r, r], rtol=1e-12)
    sq = W.uniform_grid(2, (2, 3), 4, 8)
    om2 = H.rank_one_weights(sq, 1)
    xi = np.random.default_rng(1).uniform(0, 1, (20, 2))
    for r in range(2):
        _, J = geometry.patch_map(sq, 1, xi)
        Ji = np.linalg.inv(J)
        Arr = (np.einsum("qac,qbc->qab", Ji, Ji) * np.abs(np.linalg.det(J))[:, None, None])[:, r, r]
        assert np.allclose(om2[r][0](xi[:, 0]) * om2[r][1](xi[:, 1]), Arr, rtol=1e-12)


def _rate(mg):
    A = mg.Af.toarray()
    V = np.array([mg.vcycle(e) for e in np.eye(A.shape[0])]).T
    sym = np.abs(V - V.T).max() / np.abs(V).max()
    return float(np.max(np.abs(np.linalg.eigvals(np.eye(A.shape[0]) - V @ A)))), sym


@pytest.mark.parametrize("geom", ["unit", "annulus"])
def test_vcycle_symmetric_and_robust_in_p_and_h(geom):
    rates = {}
    for p in (2, 4, 7):
        for n in (8, 16):
            dom = W.uniform_grid(2, (3, 3), p, n, W.UNIT if geom == "unit" else W.ANNULUS, None, ("vertex",))
            k = 4 if geom == "unit" else 0
            K, _, _ = assembly.assemble_patch(dom, k, with_rhs=False)
            for mask, alpha in ((0, 1e-2), (0b1111, 0.0)):
                rho, sym = _rate(H.HighOrderMG(dom, k, K, mask, alpha))
                assert sym < 1e-11
                rates[(p, n, mask)] = rho
    bound = 0.7 if geom == "unit" else 0.85
    assert max(rates.values()) < bound, rates
    # robustness: no growth with p or h beyond a few percent
    assert max(rates.values()) - min(rates.values()) < 0.1, rates


@pytest.mark.parametrize("case", ["square_p4", "annulus_p5", "uneven_p5_7"])
def test_ietidp_with_highorder_mg_equals_global_solve(case):
    if case == "square_p4":
        dom = W.random_quad_rhs(W.uniform_grid(2, (2, 2), 4, 8), seed=3)
    elif case == "annulus_p5":
        dom = W.annulus_6x6(8, 5, grid=(3, 3))
    else:
        dom = W.Domain(2, (2, 2), [[5, 7], [7, 5]], [[8, 8], [8, 16]], W.UNIT, {"kind": "sin2d"},
                       (W.PRIMAL_VERTEX, W.PRIMAL_EDGE), "uneven_ho")
        dom = W.random_quad_rhs(dom, seed=5)
    mp = Multipatch(dom)
    ref = mp.to_patches(mp.solve_global())
    s = O.IETIDP(dom, O.Options(mode="mg", mg_kind="highorder"))
    u = s.solve()
    assert s.stats.converged
    err = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(u, ref)) / sum(np.sum(b ** 2) for b in ref))
    assert err < 1e-10, err
    its = [i for i in s.stats.neumann_its if i > 0]
    print(case, "outer", s.stats.outer_it, "mean Neumann CG iterations", np.mean(its))
    assert np.mean(its) < 40, np.mean(its)


def test_highorder_mode_basis_equals_direct_basis():
    """With the high-order multigrid the primal basis is still the solution of
    Eq. 6 (computed with the standard V-cycle as the preconditioner): equal
    to the direct basis, C Phi = I and Phi K-orthogonal to ker C, on curved
    patches with a floating one at p = 4."""
    dom = W.annulus_6x6(8, 4, grid=(3, 3))
    a = O.IETIDP(dom, O.Options(mode="direct"))
    b = O.IETIDP(dom, O.Options(mode="mg", mg_kind="highorder"))
    rng = np.random.default_rng(3)
    for k in range(a.N):
        assert np.abs(a.phi[k] - b.phi[k]).max() < 1e-9
        C, phi, K = b.C[k].toarray(), b.phi[k], b.K[k]
        assert np.abs(C @ phi - np.eye(C.shape[0])).max() < 1e-12
        v = rng.standard_normal(K.shape[0])
        v -= C.T @ np.linalg.solve(C @ C.T, C @ v)
        assert np.abs(phi.T @ (K @ v)).max() < 1e-9 * np.linalg.norm(K @ v)
