"""B-spline bases on the unit interval and their tensor products (Sec. 2).

ORACLE (test infrastructure only).  Plain FP64 numpy.

* open uniform knot vectors, maximal smoothness C^{p-1}: n elements give
  n + p basis functions per direction;
* basis values and first derivatives by the Cox-de Boor recursion;
* Gauss-Legendre rules (numpy's ``leggauss``);
* the canonical embedding of a coarse spline space into its dyadic refinement
  (knot insertion, Boehm's algorithm) used as multigrid prolongation (Sec. 4).

Pins (tests/test_oracle_splines.py): partition of unity; derivative against
central differences; knot insertion reproduces coarse splines exactly at
random points; P 1 = 1; 1D integrals sum to 1.
"""
from __future__ import annotations

import numpy as np


def open_uniform_knots(n: int, p: int) -> np.ndarray:
    """Open knot vector on [0,1] with n uniform elements, degree p."""
    inner = np.arange(1, n) / n
    return np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])


def basis_funs(knots: np.ndarray, p: int, x: np.ndarray, deriv: bool = False):
    """All basis functions N_{i,p} (i = 0..m-1, m = len(knots)-p-1) at points x.

    Cox-de Boor: N_{i,0} = 1 on [t_i, t_{i+1}); N_{i,q} = w1 N_{i,q-1} +
    w2 N_{i+1,q-1} with w1 = (x - t_i)/(t_{i+q} - t_i), w2 = (t_{i+q+1} - x)/
    (t_{i+q+1} - t_{i+1}) and 0/0 := 0.  The last non-empty interval is closed
    so that x = 1 is covered.  Returns an array (len(x), m) and, when
    ``deriv``, the first derivatives too.
    """
    t = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nk = len(t)
    last = np.max(np.nonzero(t[:-1] < t[1:])[0])
    N = np.zeros((len(x), nk - 1))
    for i in range(nk - 1):
        if t[i] < t[i + 1]:
            inside = (x >= t[i]) & (x < t[i + 1])
            if i == last:
                inside |= x == t[i + 1]
            N[:, i] = inside
    levels = [N]
    for q in range(1, p + 1):
        prev = levels[-1]
        cur = np.zeros((len(x), nk - 1 - q))
        for i in range(nk - 1 - q):
            d1 = t[i + q] - t[i]
            d2 = t[i + q + 1] - t[i + 1]
            if d1 > 0:
                cur[:, i] += (x - t[i]) / d1 * prev[:, i]
            if d2 > 0:
                cur[:, i] += (t[i + q + 1] - x) / d2 * prev[:, i + 1]
        levels.append(cur)
    vals = levels[p]
    if not deriv:
        return vals
    dvals = np.zeros_like(vals)
    if p > 0:
        prev = levels[p - 1]
        for i in range(vals.shape[1]):
            d1 = t[i + p] - t[i]
            d2 = t[i + p + 1] - t[i + 1]
            if d1 > 0:
                dvals[:, i] += p / d1 * prev[:, i]
            if d2 > 0:
                dvals[:, i] -= p / d2 * prev[:, i + 1]
    return vals, dvals


def gauss_points(n_elem: int, nq: int):
    """Tensor-free 1D rule: nq Gauss-Legendre points on each of n_elem uniform
    elements of [0,1].  Returns (points, weights), element-major."""
    g, w = np.polynomial.legendre.leggauss(nq)
    h = 1.0 / n_elem
    pts = np.concatenate([(e + 0.5 * (g + 1.0)) * h for e in range(n_elem)])
    wts = np.concatenate([0.5 * w * h for _ in range(n_elem)])
    return pts, wts


def basis_integrals(n: int, p: int) -> np.ndarray:
    """int_0^1 N_{i,p} for all i, by Gauss quadrature (p+1 points per element
    integrate a degree-p polynomial exactly)."""
    x, w = gauss_points(n, p + 1)
    return w @ basis_funs(open_uniform_knots(n, p), p, x)


def insert_knot(knots: np.ndarray, p: int, tnew: float):
    """Boehm's single knot insertion.  Returns (new knots, matrix Q) with
    c_new = Q c_old for the coefficients of one and the same spline."""
    t = knots
    m = len(t) - p - 1
    k = int(np.searchsorted(t, tnew, side="right") - 1)   # t_k <= tnew < t_{k+1}
    Q = np.zeros((m + 1, m))
    for i in range(m + 1):
        if i <= k - p:
            Q[i, i] = 1.0
        elif i >= k + 1:
            Q[i, i - 1] = 1.0
        else:
            a = (tnew - t[i]) / (t[i + p] - t[i])
            Q[i, i] = a
            Q[i, i - 1] = 1.0 - a
    return np.insert(t, k + 1, tnew), Q


def refine_matrix(n_coarse: int, p: int, factor: int = 2) -> np.ndarray:
    """Prolongation P (m_fine x m_coarse) from n_coarse to factor*n_coarse
    uniform elements (same degree, maximal smoothness): the canonical
    embedding of nested spline spaces.  factor == 1 gives the identity."""
    t = open_uniform_knots(n_coarse, p)
    m = n_coarse + p
    P = np.eye(m)
    if factor == 1:
        return P
    assert factor == 2
    for e in range(n_coarse):
        t, Q = insert_knot(t, p, (e + 0.5) / n_coarse)
        P = Q @ P
    return P


def mass_1d(n: int, p: int) -> np.ndarray:
    """Dense 1D parameter-domain mass matrix int N_i N_j (exact Gauss rule)."""
    x, w = gauss_points(n, p + 1)
    B = basis_funs(open_uniform_knots(n, p), p, x)
    return B.T @ (w[:, None] * B)


def stiffness_1d(n: int, p: int) -> np.ndarray:
    """Dense 1D stiffness int N_i' N_j' (exact Gauss rule)."""
    x, w = gauss_points(n, p + 1)
    _, D = basis_funs(open_uniform_knots(n, p), p, x, deriv=True)
    return D.T @ (w[:, None] * D)
