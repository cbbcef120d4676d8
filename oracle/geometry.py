"""Patch geometry maps and right-hand sides of the model problem (Sec. 2, Eq. 1).

ORACLE (test infrastructure only).  Plain FP64 numpy.

Each patch is the image of the parameter box of its grid cell under one
global map G (Sec. 2: G(xi) = sum_i P_i N_i(xi), here either the identity or
the exact rational quarter circle times a linear radius):

* unit:    G(s) = s on the unit square / cube;
* annulus: G(s1, s2) = (1 + s2) * C(s1), with C the degree-2 NURBS quarter
           circle with control points (1,0), (1,1), (0,1) and weights
           (1, 1/sqrt 2, 1).

Pins (tests/test_oracle_assembly.py): |C| = 1 on the whole arc and its
derivative against central differences; the patch Jacobians of both maps
against central differences of the maps; the annulus right-hand side against
a finite difference Laplacian of the manufactured solution; the annulus area.
"""
from __future__ import annotations

import numpy as np

W1 = 1.0 / np.sqrt(2.0)


def circle(t):
    """Rational quadratic quarter circle and its derivative d/dt."""
    b0 = (1 - t) ** 2
    b1 = 2 * t * (1 - t)
    b2 = t ** 2
    db0 = -2 * (1 - t)
    db1 = 2 - 4 * t
    db2 = 2 * t
    W = b0 + W1 * b1 + b2
    dW = db0 + W1 * db1 + db2
    Nx = b0 * 1.0 + W1 * b1 * 1.0 + b2 * 0.0
    Ny = b0 * 0.0 + W1 * b1 * 1.0 + b2 * 1.0
    dNx = db0 + W1 * db1
    dNy = W1 * db1 + db2
    cx, cy = Nx / W, Ny / W
    dcx = (dNx * W - Nx * dW) / W ** 2
    dcy = (dNy * W - Ny * dW) / W ** 2
    return cx, cy, dcx, dcy


def patch_map(dom, k, xi):
    """Physical points and Jacobians of patch k at local parameters xi.

    xi: array (npts, d) in (0,1)^d.  Returns X (npts, d) and J (npts, d, d)
    with J[q, a, b] = d X_a / d xi_b.
    """
    d = dom.dim
    c = dom.patch_coords(k)
    s = np.empty_like(xi)
    scale = np.empty(d)
    for r in range(d):
        scale[r] = 1.0 / dom.grid[r]
        s[:, r] = (c[r] + xi[:, r]) * scale[r]
    npts = xi.shape[0]
    if dom.geometry == "unit":
        X = s.copy()
        J = np.zeros((npts, d, d))
        for r in range(d):
            J[:, r, r] = scale[r]
        return X, J
    if dom.geometry == "annulus":
        assert d == 2
        cx, cy, dcx, dcy = circle(s[:, 0])
        rad = 1.0 + s[:, 1]
        X = np.stack([rad * cx, rad * cy], axis=1)
        J = np.zeros((npts, 2, 2))
        J[:, 0, 0] = rad * dcx * scale[0]
        J[:, 1, 0] = rad * dcy * scale[0]
        J[:, 0, 1] = cx * scale[1]
        J[:, 1, 1] = cy * scale[1]
        return X, J
    raise ValueError(dom.geometry)


def rhs_values(dom, X):
    """f at physical points X (npts, d) for the analytic right-hand sides."""
    kind = dom.rhs["kind"]
    pi = np.pi
    if kind == "sin2d":
        return 2 * pi ** 2 * np.sin(pi * X[:, 0]) * np.sin(pi * X[:, 1])
    if kind == "sin3d":
        return 3 * pi ** 2 * np.sin(pi * X[:, 0]) * np.sin(pi * X[:, 1]) * np.sin(pi * X[:, 2])
    if kind == "annulus":
        x, y = X[:, 0], X[:, 1]
        r = np.sqrt(x * x + y * y)
        s = np.sin(pi * x) * np.sin(pi * y)
        g = (r - 1) * (2 - r)
        gp = 3 - 2 * r
        return (2 * pi ** 2 * s * g
                - 2 * pi * (gp / r) * (x * np.cos(pi * x) * np.sin(pi * y)
                                       + y * np.sin(pi * x) * np.cos(pi * y))
                - s * (3 / r - 4))
    if kind == "modes":
        f = np.zeros(X.shape[0])
        for a, kk, ll in zip(dom.rhs["a"], dom.rhs["k"], dom.rhs["l"]):
            f += a * np.sin(kk * pi * X[:, 0]) * np.sin(ll * pi * X[:, 1])
        return f
    raise ValueError(kind)


def exact_solution(dom, X):
    """Manufactured solutions for the analytic right-hand sides (or None)."""
    kind = dom.rhs["kind"]
    pi = np.pi
    if kind == "sin2d":
        return np.sin(pi * X[:, 0]) * np.sin(pi * X[:, 1])
    if kind == "sin3d":
        return np.sin(pi * X[:, 0]) * np.sin(pi * X[:, 1]) * np.sin(pi * X[:, 2])
    if kind == "annulus":
        r = np.sqrt(X[:, 0] ** 2 + X[:, 1] ** 2)
        return np.sin(pi * X[:, 0]) * np.sin(pi * X[:, 1]) * (r - 1) * (2 - r)
    return None
