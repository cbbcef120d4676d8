"""Pin of the D-MG local Neumann solve reading (the banded-Cholesky route of
the CUDA path, Sec. 3.3 / Eq. 7), on the CPU.

The CUDA path solves K z = P^T g with P = I - Phi C by a Cholesky factor of
K in which, on a floating patch, one interior function (the centre of the
tensor grid) is pinned (identity row and column), and returns w = P z.  The
reading holds because P^T g is orthogonal to the constants (ker K) once that
is made exact, so the pinned system yields one solution of K z = P^T g, and
P removes the constant in which the solutions differ.  Here that route,
written with dense numpy linear algebra, must give the minimiser of Eq. 7
that the oracle computes with the sparse LU of the saddle-point matrix
[K C^T; C 0] -- on floating and non-floating patches, 2D and 3D.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ietidp as O
from paper_1705_04531_gb300 import workloads as W

DOMS = {
    "grid3x3_floating": lambda: W.uniform_grid(2, (3, 3), 3, 8, W.UNIT, None, ("vertex", "edge")),
    "annulus3x3": lambda: W.annulus_6x6(8, 2, grid=(3, 3)),
    "grid3x3x3_floating": lambda: W.uniform_grid(3, (3, 3, 3), 2, 2, W.UNIT, None, ("vertex", "edge", "face")),
}


def _pinned_route(s, k, g):
    K = s.K[k].toarray()
    C = s.C[k].toarray()
    phi = s.phi[k]
    b = g - C.T @ (phi.T @ g)                 # P^T g
    if s.floating[k]:
        b = b - b.mean()                      # exactly orthogonal to ker K
        m = s.m[k]
        centre = m[0] // 2 + m[0] * (m[1] // 2 + (m[1] * (m[2] // 2) if len(m) == 3 else 0))
        p = int(s.inv[k][centre])             # the pinned function in free numbering
        assert p >= 0
        K = K.copy()
        K[p, :] = 0.0
        K[:, p] = 0.0
        K[p, p] = 1.0
        b = b.copy()
        b[p] = 0.0
    z = sla.cho_solve(sla.cho_factor(K), b)
    return z - phi @ (C @ z)                  # w = P z


@pytest.mark.parametrize("name", list(DOMS))
def test_pinned_cholesky_route_equals_saddle_lu(name):
    s = O.IETIDP(DOMS[name](), O.Options(mode="direct"))
    rng = np.random.default_rng(7)
    nfloat = 0
    for k in range(s.N):
        g = rng.standard_normal(len(s.free[k]))
        ref = s.delta_solve(k, g)
        got = _pinned_route(s, k, g)
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), (name, k)
        nfloat += bool(s.floating[k])
    if "floating" in name:
        assert nfloat >= 1


def test_pin_without_projection_fails_on_floating_patch():
    """The two steps the reading adds are both needed: without making the
    right-hand side orthogonal to the constants the pinned solve answers a
    different problem (its result differs from the minimiser)."""
    s = O.IETIDP(DOMS["grid3x3_floating"](), O.Options(mode="direct"))
    k = [i for i in range(s.N) if s.floating[i]][0]
    rng = np.random.default_rng(8)
    g = rng.standard_normal(len(s.free[k])) + 1.0          # a constant component
    ref = s.delta_solve(k, g)
    K = s.K[k].toarray()
    m = s.m[k]
    p = int(s.inv[k][m[0] // 2 + m[0] * (m[1] // 2)])
    K[p, :] = 0.0
    K[:, p] = 0.0
    K[p, p] = 1.0
    b = g.copy()                                            # no P^T, no mean removal
    b[p] = 0.0
    z = sla.cho_solve(sla.cho_factor(K), b)
    C, phi = s.C[k].toarray(), s.phi[k]
    bad = z - phi @ (C @ z)
    assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()
