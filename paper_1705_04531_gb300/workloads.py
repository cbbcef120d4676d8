"""Seeded synthetic inputs for the inexact IETI-DP solver.

This module only *describes* problems: patch grids, degrees, element counts,
geometry kind, the right-hand side and the primal constraint set.  It holds no
arithmetic of the method (no spline evaluation, no assembly, no solver step),
so that the CPU oracle and the CUDA path can both read the same inputs while
sharing no computational code.

Domains are grids of patches (Sec. 2: a multipatch domain is a union of
non-overlapping patches, each the image of the unit square/cube).  Patch
``k = i + Px*(j + Py*l)`` covers the parameter box
``[i/Px,(i+1)/Px] x [j/Py,(j+1)/Py] (x [l/Pz,(l+1)/Pz])`` of a global map.
Degree and element count are given per patch *column* along each direction,
so every interface carries the same tangential spline space on both sides
(conforming tearing, Sec. 2).

Right-hand sides (model problem of Eq. 1, -Laplace u = f, homogeneous
Dirichlet data on the whole boundary):

* ``sin2d``   f = 2 pi^2 sin(pi x) sin(pi y)          (u = sin sin)
* ``annulus`` f = -Laplace of u = sin(pi x) sin(pi y) (r-1)(2-r)
* ``sin3d``   f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) (u = sin sin sin)
* ``modes``   f = sum_j a_j sin(k_j pi x) sin(l_j pi y)
* ``quad``    f given at the tensor grid of Gauss points of every patch
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# geometry kinds
UNIT = "unit"          # identity map of the unit square / cube, split into a grid
ANNULUS = "annulus"    # quarter annulus r in [1,2], exact NURBS map, angle along xi_1

PRIMAL_VERTEX = "vertex"
PRIMAL_EDGE = "edge"
PRIMAL_FACE = "face"


@dataclass
class Domain:
    dim: int
    grid: tuple                      # patches per direction
    degree: list                     # degree[r][c]: degree along direction r of patch column c
    nelem: list                      # nelem[r][c]: elements along direction r of patch column c
    geometry: str = UNIT
    rhs: dict = field(default_factory=lambda: {"kind": "sin2d"})
    primal: tuple = (PRIMAL_VERTEX,)
    name: str = ""

    @property
    def npatch(self) -> int:
        return int(np.prod(self.grid))

    def patch_coords(self, k: int) -> tuple:
        c = []
        for r in range(self.dim):
            c.append(k % self.grid[r])
            k //= self.grid[r]
        return tuple(c)

    def patch_degree(self, k: int) -> tuple:
        c = self.patch_coords(k)
        return tuple(int(self.degree[r][c[r]]) for r in range(self.dim))

    def patch_nelem(self, k: int) -> tuple:
        c = self.patch_coords(k)
        return tuple(int(self.nelem[r][c[r]]) for r in range(self.dim))

    def patch_ndof(self, k: int) -> int:
        return int(np.prod([n + p for n, p in zip(self.patch_nelem(k), self.patch_degree(k))]))

    def quad_shape(self, k: int) -> tuple:
        """Gauss-point grid of patch k: nelem*(degree+1) points per direction."""
        return tuple(n * (p + 1) for n, p in zip(self.patch_nelem(k), self.patch_degree(k)))


def uniform_grid(dim, grid, p, n, geometry=UNIT, rhs=None, primal=(PRIMAL_VERTEX,), name=""):
    degree = [[p] * grid[r] for r in range(dim)]
    nelem = [[n] * grid[r] for r in range(dim)]
    if rhs is None:
        rhs = {"kind": "sin2d" if dim == 2 else "sin3d"}
    return Domain(dim, tuple(grid), degree, nelem, geometry, rhs, tuple(primal), name)


# ---------------------------------------------------------------------------
# The five workload shapes (unit square 2x2 p=2; quarter annulus 6x6 p=3;
# uneven 8x8 batch; unit cube 2x2x2 p=2; serving stream).  ``scale`` shrinks
# the element counts for tests that must finish quickly on the CPU oracle.
# ---------------------------------------------------------------------------

def square_2x2(n=16, p=2):
    return uniform_grid(2, (2, 2), p, n, UNIT, {"kind": "sin2d"}, (PRIMAL_VERTEX,),
                        f"square2x2_p{p}_n{n}")


def annulus_6x6(n=64, p=3, grid=(6, 6)):
    return uniform_grid(2, grid, p, n, ANNULUS, {"kind": "annulus"},
                        (PRIMAL_VERTEX, PRIMAL_EDGE), f"annulus{grid[0]}x{grid[1]}_p{p}_n{n}")


def cube_2x2x2(n=32, p=2):
    return uniform_grid(3, (2, 2, 2), p, n, UNIT, {"kind": "sin3d"},
                        (PRIMAL_VERTEX, PRIMAL_EDGE, PRIMAL_FACE), f"cube2x2x2_p{p}_n{n}")


def uneven_8x8(seed=0, grid=(8, 8), degrees=(2, 3, 4), nelems=(32, 64, 128, 256)):
    """Uneven batch: degree and element count drawn per patch column (x) and
    per patch row (y) so that every interface matches; then f ~ U(-1,1) at
    the Gauss points, patch by patch, each patch's point grid x-fastest.

    Draw order with ``numpy.random.default_rng(seed)``: x-columns (degrees,
    then element counts), y-rows (degrees, then element counts), then f.
    """
    rng = np.random.default_rng(seed)
    px = rng.choice(np.asarray(degrees), size=grid[0])
    nx = rng.choice(np.asarray(nelems), size=grid[0])
    py = rng.choice(np.asarray(degrees), size=grid[1])
    ny = rng.choice(np.asarray(nelems), size=grid[1])
    dom = Domain(2, tuple(grid), [list(map(int, px)), list(map(int, py))],
                 [list(map(int, nx)), list(map(int, ny))], UNIT, {"kind": "quad"},
                 (PRIMAL_VERTEX, PRIMAL_EDGE), f"uneven{grid[0]}x{grid[1]}_s{seed}")
    values = []
    for k in range(dom.npatch):
        qs = dom.quad_shape(k)
        values.append(rng.uniform(-1.0, 1.0, size=int(np.prod(qs))))
    dom.rhs = {"kind": "quad", "values": values}
    return dom


def sine_modes_rhs(rng, nmodes=8):
    a = rng.uniform(-1.0, 1.0, size=nmodes)
    k = rng.integers(1, 5, size=nmodes)
    l = rng.integers(1, 5, size=nmodes)
    return {"kind": "modes", "a": [float(v) for v in a], "k": [int(v) for v in k],
            "l": [int(v) for v in l]}


@dataclass
class Request:
    rid: int
    arrival: float
    domain: Domain


def serving_stream(nreq=512, rate=100.0, seed=0, ms=(2, 4, 6, 8), ps=(2, 3),
                   ns=(16, 32, 64, 128)):
    """Poisson arrivals of 2D Poisson requests on an m x m grid of the unit
    square: m, p, n drawn per request, f a sum of 8 random sine modes."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(nreq):
        t += rng.exponential(1.0 / rate)
        m = int(rng.choice(ms))
        p = int(rng.choice(ps))
        n = int(rng.choice(ns))
        rhs = sine_modes_rhs(rng)
        dom = uniform_grid(2, (m, m), p, n, UNIT, rhs, (PRIMAL_VERTEX, PRIMAL_EDGE),
                           f"req{i}_m{m}_p{p}_n{n}")
        out.append(Request(i, t, dom))
    return out


def random_quad_rhs(dom: Domain, seed: int = 1) -> Domain:
    """Replace f by U(-1,1) values at every patch's Gauss points (no symmetry,
    so the dual problem is never trivial)."""
    rng = np.random.default_rng(seed)
    vals = [rng.uniform(-1.0, 1.0, size=int(np.prod(dom.quad_shape(k)))) for k in range(dom.npatch)]
    dom.rhs = {"kind": "quad", "values": vals}
    dom.name = dom.name + f"_rq{seed}"
    return dom


def by_name(name: str, scale: Optional[int] = None) -> Domain:
    """Workloads by descriptive name; ``scale`` divides element counts."""
    s = scale or 1
    if name == "square2x2_p2_n16":
        return square_2x2(16 // s if s > 1 else 16, 2)
    if name == "annulus6x6_p3_n64":
        return annulus_6x6(max(4, 64 // s), 3)
    if name == "cube2x2x2_p2_n32":
        return cube_2x2x2(max(4, 32 // s), 2)
    if name in ("annulus6x6_p4_n32", "annulus6x6_p7_n32"):
        return annulus_6x6(max(4, 32 // s), int(name[len("annulus6x6_p")]))
    if name == "uneven8x8_s0":
        if s == 1:
            return uneven_8x8(0)
        return uneven_8x8(0, nelems=tuple(max(4, v // s) for v in (32, 64, 128, 256)))
    raise KeyError(name)
