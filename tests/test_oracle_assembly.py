"""Pins of the per-patch Galerkin assembly (Eq. 1; parameter mass of
Sec. 3.2) and the geometry maps (Sec. 2)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assembly, geometry, splines
from oracle.multigrid import Hierarchy
from paper_1705_04531_gb300 import workloads as W


def test_circle_is_exact():
    t = np.linspace(0, 1, 101)
    cx, cy, dcx, dcy = geometry.circle(t)
    assert np.allclose(cx ** 2 + cy ** 2, 1.0, atol=1e-15)
    h = 1e-6
    a = geometry.circle(t[1:-1] + h)
    b = geometry.circle(t[1:-1] - h)
    assert np.allclose(dcx[1:-1], (a[0] - b[0]) / (2 * h), atol=1e-8)
    assert np.allclose(dcy[1:-1], (a[1] - b[1]) / (2 * h), atol=1e-8)


@pytest.mark.parametrize("dom", [W.annulus_6x6(4, 3, grid=(3, 2)), W.cube_2x2x2(2, 2)])
def test_patch_jacobian_vs_differences(dom):
    rng = np.random.default_rng(3)
    h = 1e-6
    for k in (0, dom.npatch - 1):
        xi = rng.uniform(0.05, 0.95, (20, dom.dim))
        _, J = geometry.patch_map(dom, k, xi)
        for b in range(dom.dim):
            e = np.zeros(dom.dim)
            e[b] = h
            Xp, _ = geometry.patch_map(dom, k, xi + e)
            Xm, _ = geometry.patch_map(dom, k, xi - e)
            assert np.allclose(J[:, :, b], (Xp - Xm) / (2 * h), atol=1e-8)


def test_annulus_rhs_is_minus_laplacian():
    dom = W.annulus_6x6(4, 3)
    rng = np.random.default_rng(0)
    th = rng.uniform(0.05, np.pi / 2 - 0.05, 30)
    r = rng.uniform(1.05, 1.95, 30)
    X = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    h = 1e-4
    lap = np.zeros(30)
    for a in range(2):
        e = np.zeros(2)
        e[a] = h
        lap += (geometry.exact_solution(dom, X + e) - 2 * geometry.exact_solution(dom, X)
                + geometry.exact_solution(dom, X - e)) / h ** 2
    assert np.allclose(geometry.rhs_values(dom, X), -lap, atol=2e-5)


@pytest.mark.parametrize("dom", [W.square_2x2(4, 2), W.annulus_6x6(4, 3), W.cube_2x2x2(2, 2),
                                 W.uneven_8x8(0, grid=(2, 2), nelems=(2, 4))])
def test_stiffness_kernel_mass_sum_symmetry(dom):
    for k in range(dom.npatch):
        K, f, M = assembly.assemble_patch(dom, k)
        one = np.ones(K.shape[0])
        assert np.abs(K @ one).max() < 1e-12 * abs(K).max()
        assert abs((K - K.T)).max() < 1e-13 * abs(K).max()
        assert abs(M.sum() - 1.0) < 1e-13
        assert abs((M - M.T)).max() < 1e-16


def test_annulus_area():
    dom = W.annulus_6x6(2, 2)
    area = 0.0
    for k in range(dom.npatch):
        tabs = assembly.patch_tables(dom, k)
        xi, w = assembly.quad_grid(dom, k, tabs)
        _, J = geometry.patch_map(dom, k, xi)
        area += np.sum(w * np.abs(np.linalg.det(J)))
    # the NURBS map is exact but rational: 3 Gauss points per element
    assert abs(area - 0.75 * np.pi) < 1e-6


def test_unit_square_is_kronecker():
    dom = W.square_2x2(4, 3)
    K, _, _ = assembly.assemble_patch(dom, 0)
    K1 = sp.csr_matrix(splines.stiffness_1d(4, 3))
    M1 = sp.csr_matrix(splines.mass_1d(4, 3))
    ref = sp.kron(M1, K1) + sp.kron(K1, M1)       # patch size cancels in 2D
    assert abs(K - ref).max() < 1e-12


def test_galerkin_equals_rediscretization():
    fine = W.square_2x2(8, 2)
    coarse = W.square_2x2(4, 2)
    Kf, _, _ = assembly.assemble_patch(fine, 1)
    Kc, _, _ = assembly.assemble_patch(coarse, 1)
    h = Hierarchy(Kf, (8, 8), (2, 2), cmin=4)
    assert h.L == 2
    assert abs(h.K[0] - Kc).max() < 1e-12
    assert abs(h.P[1].T @ h.M[1] @ h.P[1] - h.M[0]).max() < 1e-15


def test_load_integrates_f():
    """sum_i f_i = int f (partition of unity), against a fine Gauss rule."""
    dom = W.square_2x2(8, 2)
    _, f, _ = assembly.assemble_patch(dom, 3)
    x, w = splines.gauss_points(64, 6)
    X = 0.5 + 0.5 * x
    # f = 2 pi^2 sin(pi x) sin(pi y) on [1/2,1]^2, scaled weights
    g = 2 * np.pi ** 2 * np.outer(np.sin(np.pi * X), np.sin(np.pi * X))
    ref = 0.25 * w @ g @ w
    assert abs(f.sum() - ref) < 1e-5


@pytest.mark.parametrize("dom", [W.annulus_6x6(4, 3, grid=(2, 2)),
                                 W.random_quad_rhs(W.uneven_8x8(0, grid=(2, 2), nelems=(4, 8))),
                                 W.cube_2x2x2(3, 2)])
def test_single_row_equals_full_assembly(dom):
    """The one-row oracle used for full-size checks equals the rows of the
    full patch assembly (same Gauss rule, support-restricted)."""
    for k in range(dom.npatch):
        K, f, _ = assembly.assemble_patch(dom, k)
        rng = np.random.default_rng(k)
        for i in rng.integers(0, K.shape[0], 4):
            cols, vals, fi = assembly.row_stiffness_load(dom, k, int(i))
            ref = K[int(i)].toarray().ravel()
            got = np.zeros_like(ref)
            got[cols] = vals
            assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
            assert abs(fi - f[int(i)]) <= 1e-12 * max(1.0, abs(f[int(i)]))
