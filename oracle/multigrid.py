"""Geometric h-multigrid for one patch (Sec. 4: nested grids, p fixed,
canonical embedding/restriction, Gauss-Seidel smoothing) and PCG.

ORACLE (test infrastructure only).  Plain FP64 numpy/scipy.

Readings of the paper used here (the paper names the ingredients only):

* levels: every direction with more than ``cmin`` (=4) elements and an even
  element count is halved, until none is; the coarsest level is solved by a
  dense Cholesky factorization;
* transfers: P = P_d x ... x P_1 from 1D knot insertion, restriction P^T;
* coarse operators: Galerkin K_{l-1} = P^T K_l P on the full tensor grid;
  Dirichlet or interface dofs are removed on every level by a side mask
  (masked Galerkin equals Galerkin of the masked operator because P maps
  coarse interior functions to fine functions vanishing on the boundary);
* regularization K_M = K + alpha M^ with alpha = 1e-2 for patches whose
  boundary does not touch the Dirichlet boundary (Sec. 3.2), with the
  parameter mass of each level (equal to its Galerkin coarsening);
* smoother: "standard Gauss-Seidel" read as multicolor Gauss-Seidel with
  (p_1+1)...(p_d+1) colors, color(i) = sum_r (i_r mod (p_r+1)) * stride_r;
  pre-smoothing sweeps the colors upwards, post-smoothing downwards, so the
  V-cycle is a symmetric preconditioner; nu_1 = nu_2 = 2.

Pins (tests/test_oracle_domain_mg.py): the V-cycle operator is symmetric and
its error operator contracts at the same rate (< 0.3) on two mesh sizes; a
V-cycle on a 1-level hierarchy is the exact solve; the rows of one color do
not couple (so the color order alone fixes the smoother); PCG with it matches
a sparse direct solve, also on a floating (regularised) patch.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import splines


def coarsening_schedule(nelem, cmin=4):
    """Element counts per level, coarsest first."""
    sched = [tuple(nelem)]
    while True:
        cur = sched[-1]
        nxt = tuple(n // 2 if (n > cmin and n % 2 == 0) else n for n in cur)
        if nxt == cur:
            break
        sched.append(nxt)
    return sched[::-1]


def _kron_all(mats):
    out = mats[0]
    for M in mats[1:]:
        out = sp.kron(M, out, format="csr")
    return sp.csr_matrix(out)


def tensor_index(m, idx):
    """Per-direction indices of flat tensor indices (first direction fastest)."""
    out = []
    for mr in m:
        out.append(idx % mr)
        idx = idx // mr
    return out


def free_mask(m, side_mask):
    """Boolean over the tensor grid: False on the dofs of masked sides.
    Side 2r is the lower end of direction r, side 2r+1 the upper end."""
    n = int(np.prod(m))
    ti = tensor_index(m, np.arange(n))
    ok = np.ones(n, dtype=bool)
    for r in range(len(m)):
        if side_mask >> (2 * r) & 1:
            ok &= ti[r] != 0
        if side_mask >> (2 * r + 1) & 1:
            ok &= ti[r] != m[r] - 1
    return ok


class Hierarchy:
    """Galerkin hierarchy of one patch's full-grid stiffness (unmasked)."""

    def __init__(self, K_fine, nelem, degree, cmin=4):
        self.degree = tuple(degree)
        self.sched = coarsening_schedule(nelem, cmin)
        self.L = len(self.sched)
        self.m = [tuple(n + p for n, p in zip(ne, degree)) for ne in self.sched]
        self.P = [None] * self.L       # P[l]: level l-1 -> level l
        for l in range(1, self.L):
            mats = []
            for r in range(len(degree)):
                fac = self.sched[l][r] // self.sched[l - 1][r]
                mats.append(sp.csr_matrix(splines.refine_matrix(self.sched[l - 1][r], degree[r], fac)))
            self.P[l] = _kron_all(mats)
        self.K = [None] * self.L
        self.K[-1] = sp.csr_matrix(K_fine)
        for l in range(self.L - 1, 0, -1):
            self.K[l - 1] = sp.csr_matrix(self.P[l].T @ self.K[l] @ self.P[l])
        self.M = [_kron_all([sp.csr_matrix(splines.mass_1d(n, p)) for n, p in zip(ne, degree)])
                  for ne in self.sched]


class MGOperator:
    """V-cycle preconditioner for (K + alpha M^) restricted to unmasked dofs."""

    def __init__(self, hier: Hierarchy, side_mask: int, alpha: float = 0.0, nu1=2, nu2=2):
        self.h = hier
        self.nu1, self.nu2 = nu1, nu2
        L = hier.L
        self.free = [np.nonzero(free_mask(hier.m[l], side_mask))[0] for l in range(L)]
        self.A = []
        self.Pf = [None] * L
        self.colors = []
        for l in range(L):
            Al = hier.K[l] + alpha * hier.M[l] if alpha else hier.K[l]
            fr = self.free[l]
            self.A.append(sp.csr_matrix(Al[fr][:, fr]))
            if l > 0:
                self.Pf[l] = sp.csr_matrix(hier.P[l][fr][:, self.free[l - 1]])
            ti = tensor_index(hier.m[l], fr)
            col = np.zeros(len(fr), dtype=np.int64)
            stride = 1
            for r, p in enumerate(hier.degree):
                col += (ti[r] % (p + 1)) * stride
                stride *= p + 1
            groups = []
            for c in range(stride):
                idx = np.nonzero(col == c)[0]
                groups.append((idx, sp.csr_matrix(self.A[l][idx]), self.A[l].diagonal()[idx]))
            self.colors.append(groups)
        A0 = self.A[0].toarray()
        self.chol0 = sla.cho_factor(A0) if A0.size else None

    def sweep(self, l, x, b, forward):
        groups = self.colors[l] if forward else self.colors[l][::-1]
        for idx, Arows, dg in groups:
            if len(idx) == 0:
                continue
            x[idx] += (b[idx] - Arows @ x) / dg

    def vcycle(self, b, l=None):
        if l is None:
            l = self.h.L - 1
        if l == 0:
            if self.chol0 is None:
                return np.zeros(0)
            return sla.cho_solve(self.chol0, b)
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            self.sweep(l, x, b, True)
        r = b - self.A[l] @ x
        xc = self.vcycle(self.Pf[l].T @ r, l - 1)
        x += self.Pf[l] @ xc
        for _ in range(self.nu2):
            self.sweep(l, x, b, False)
        return x


def pcg(apply_A, b, precond, tol, maxit=500, project=None):
    """Preconditioned CG, x0 = 0, stop when ||r|| <= tol ||b||.

    ``project`` (optional) is applied to the preconditioned residual (used for
    the null-space method on ker C).  Returns (x, iterations, converged)."""
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, True
    r = b.copy()
    z = precond(r)
    if project is not None:
        z = project(z)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= tol * nb:
            return x, it, True
        z = precond(r)
        if project is not None:
            z = project(z)
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, maxit, False
