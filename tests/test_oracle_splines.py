"""Pins of the spline oracle (Sec. 2: Cox-de Boor bases; Sec. 4: canonical
embedding of nested spline spaces) against facts that hold independently of
it: partition of unity, derivatives by differences, exact reproduction under
knot insertion, Gauss exactness, closed-form basis integrals."""
import numpy as np
import pytest

from oracle import splines


@pytest.mark.parametrize("n,p", [(1, 1), (4, 2), (7, 3), (8, 4)])
def test_partition_of_unity(n, p):
    x = np.random.default_rng(0).uniform(0, 1, 50)
    x = np.concatenate([x, [0.0, 1.0]])
    B = splines.basis_funs(splines.open_uniform_knots(n, p), p, x)
    assert B.shape == (len(x), n + p)
    assert np.allclose(B.sum(1), 1.0, atol=1e-14)
    assert (B >= -1e-15).all()


@pytest.mark.parametrize("n,p", [(4, 2), (5, 3), (8, 4)])
def test_derivative_vs_differences(n, p):
    t = splines.open_uniform_knots(n, p)
    x = np.random.default_rng(1).uniform(0.01, 0.99, 20)
    h = 1e-6
    _, D = splines.basis_funs(t, p, x, deriv=True)
    fd = (splines.basis_funs(t, p, x + h) - splines.basis_funs(t, p, x - h)) / (2 * h)
    assert np.allclose(D, fd, atol=1e-6 * n)


@pytest.mark.parametrize("n,p", [(2, 1), (4, 2), (4, 3), (8, 4), (1, 2)])
def test_knot_insertion_reproduces_splines(n, p):
    rng = np.random.default_rng(2)
    P = splines.refine_matrix(n, p)
    c = rng.standard_normal(n + p)
    x = rng.uniform(0, 1, 100)
    coarse = splines.basis_funs(splines.open_uniform_knots(n, p), p, x) @ c
    fine = splines.basis_funs(splines.open_uniform_knots(2 * n, p), p, x) @ (P @ c)
    assert np.allclose(coarse, fine, atol=1e-13)
    assert np.allclose(P.sum(1), 1.0, atol=1e-15)      # P 1 = 1
    assert P.shape == (2 * n + p, n + p)


@pytest.mark.parametrize("n,p", [(4, 2), (6, 3), (9, 4)])
def test_basis_integrals_closed_form(n, p):
    t = splines.open_uniform_knots(n, p)
    closed = np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(n + p)])
    q = splines.basis_integrals(n, p)
    assert np.allclose(q, closed, atol=1e-15)
    assert abs(q.sum() - 1.0) < 1e-14


def test_gauss_exactness():
    for nq in (1, 2, 3, 5):
        x, w = splines.gauss_points(3, nq)
        for k in range(2 * nq):
            assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-14


def test_stiffness_1d_p1_textbook():
    n = 5
    K = splines.stiffness_1d(n, 1)
    h = 1.0 / n
    T = (np.diag(np.full(n + 1, 2.0)) - np.diag(np.ones(n), 1) - np.diag(np.ones(n), -1)) / h
    T[0, 0] = T[-1, -1] = 1.0 / h
    assert np.allclose(K, T, atol=1e-12)
