"""Primal basis (Eq. 6) by CG with the Schoeberl-Zulehner preconditioner
(Sec. 3.2), the paper's route for the MG set-up.

ORACLE (test infrastructure only).  Plain FP64 numpy on top of the MG
hierarchies of ``oracle.ietidp.IETIDP`` (mode "mg").

For patch k and primal row j, Eq. 6 is the saddle-point system

    [ K  C^T ] [phi_j]   [ 0   ]
    [ C  0   ] [mu_j ] = [ e_j ].

Building blocks (Sec. 3.2): Khat^{-1} = a multigrid V-cycle on the
regularized matrix K_M = K + 1e-2 M^ (K on patches with a Dirichlet side),
and Hhat = 0.99 H with H = C Khat^{-1} C^T computed exactly (n_Pi^(k)
V-cycles).  The SZ preconditioner

    P = [ Khat  C^T                 ]
        [ C     C Khat^{-1} C^T - Hhat ]

is applied as w1 = Khat^{-1} r1, z2 = Hhat^{-1} (C w1 - r2),
z1 = w1 - W z2 with W = Khat^{-1} C^T (precomputed).  When Khat > K and
Hhat < C Khat^{-1} C^T, P^{-1} [K C^T; C 0] is self-adjoint and positive
definite in the inner product of D = P - [K C^T; C 0]
= diag(Khat - K, C Khat^{-1} C^T - Hhat), so plain CG applies; every D
product is formed from available quantities: <r, r>_D = r.rt - r.(A r) with
rt the unpreconditioned residual (P r = rt).  One Khat^{-1} and one product
with the saddle matrix per step.

Reading (the paper gives Hhat = 0.99 H but no scaling of Khat): Khat^{-1} =
0.99 V.  One symmetric V-cycle satisfies V <= K_M^{-1} <= K^{-1}; the factor
makes Khat - K strictly positive also where the V-cycle is nearly exact.
The iteration stops when <r, r>_D has dropped by tol_basis^2.

Pins (tests/test_oracle_szcg.py): the basis equals the direct solution of
Eq. 6 (C phi = I, phi^T K v = 0 on ker C); D is positive definite and the
preconditioned matrix D-self-adjoint (dense, tiny patch); iteration counts
below those of the null-space CG of R10.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

KHAT_SCALE = 0.99
HHAT_SCALE = 0.99


class SZPatch:
    """SZ building blocks of one patch: Khat^{-1}, W = Khat^{-1} C^T, Hhat^{-1}."""

    def __init__(self, s, k):
        self.s, self.k = s, k
        self.K = s.K[k]
        self.C = s.C[k].toarray()
        self.mg = s.mgN[k]
        npi = self.C.shape[0]
        self.W = np.column_stack([self.khat_inv(self.C[j]) for j in range(npi)]) if npi else np.zeros((len(s.free[k]), 0))
        H = self.C @ self.W
        self.H = 0.5 * (H + H.T)
        self.Hhat_chol = sla.cho_factor(HHAT_SCALE * self.H) if npi else None

    def khat_inv(self, r):
        return KHAT_SCALE * self.mg.vcycle(r)

    def hhat_inv(self, r2):
        return sla.cho_solve(self.Hhat_chol, r2)

    def precond(self, r1, r2):
        w1 = self.khat_inv(r1)
        z2 = self.hhat_inv(self.C @ w1 - r2)
        return w1 - self.W @ z2, z2

    def saddle(self, y1, y2):
        return self.K @ y1 + self.C.T @ y2, self.C @ y1


def sz_basis_column(pz: SZPatch, j, tol, maxit):
    """phi_j by SZ-preconditioned CG.  Returns (phi_j, iterations, converged).

    The recursively updated residuals drift by rounding (r.rt - r.(A r) is a
    difference of close numbers at tol_basis = 1e-12), so the iteration
    restarts from the residual b - A x after every 1e-4 of reduction."""
    n, npi = pz.W.shape
    b1, b2 = np.zeros(n), np.zeros(npi)
    b2[j] = 1.0
    x1, x2 = np.zeros(n), np.zeros(npi)
    rt1, rt2 = b1.copy(), b2.copy()
    r1, r2 = pz.precond(rt1, rt2)
    Ar1, Ar2 = pz.saddle(r1, r2)
    rho = r1 @ rt1 + r2 @ rt2 - (r1 @ Ar1 + r2 @ Ar2)
    rho0 = rho
    rho_cycle = rho
    restarts = 0
    p1, p2, Ap1, Ap2 = r1.copy(), r2.copy(), Ar1.copy(), Ar2.copy()
    for it in range(1, maxit + 1):
        q1, q2 = pz.precond(Ap1, Ap2)
        sigma = p1 @ Ap1 + p2 @ Ap2 - (q1 @ Ap1 + q2 @ Ap2)
        if sigma <= 0.0:
            return x1, it, False
        alpha = rho / sigma
        x1 += alpha * p1
        x2 += alpha * p2
        rt1 -= alpha * Ap1
        rt2 -= alpha * Ap2
        r1 -= alpha * q1
        r2 -= alpha * q2
        Aq1, Aq2 = pz.saddle(q1, q2)
        Ar1 -= alpha * Aq1
        Ar2 -= alpha * Aq2
        rho_new = r1 @ rt1 + r2 @ rt2 - (r1 @ Ar1 + r2 @ Ar2)
        if 0.0 <= rho_new <= tol * tol * rho0:
            return x1, it, True
        if (rho_new <= 1e-8 * rho_cycle or rho_new < 0.0) and restarts < 20:
            restarts += 1
            t1, t2 = pz.saddle(x1, x2)
            rt1, rt2 = b1 - t1, b2 - t2
            r1, r2 = pz.precond(rt1, rt2)
            Ar1, Ar2 = pz.saddle(r1, r2)
            rho = r1 @ rt1 + r2 @ rt2 - (r1 @ Ar1 + r2 @ Ar2)
            rho_cycle = rho
            if rho <= tol * tol * rho0:
                return x1, it, True
            p1, p2, Ap1, Ap2 = r1.copy(), r2.copy(), Ar1.copy(), Ar2.copy()
            continue
        beta = rho_new / rho
        rho = rho_new
        p1 = r1 + beta * p1
        p2 = r2 + beta * p2
        Ap1 = Ar1 + beta * Ap1
        Ap2 = Ar2 + beta * Ap2
    return x1, maxit, False


def sz_basis(s, tol=None, maxit=None):
    """Primal basis of every patch by SZ-CG.  Returns (list of n x n_Pi arrays,
    list of iteration counts)."""
    tol = s.o.tol_basis if tol is None else tol
    maxit = s.o.maxit_inner if maxit is None else maxit
    phis, its = [], []
    for k in range(s.N):
        pz = SZPatch(s, k)
        npi = pz.W.shape[1]
        cols = []
        for j in range(npi):
            c, it, ok = sz_basis_column(pz, j, tol, maxit)
            cols.append(c)
            its.append(it)
        phis.append(np.column_stack(cols) if cols else np.zeros((pz.W.shape[0], 0)))
    return phis, its
