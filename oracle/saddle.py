"""MG-MG-S variant: Bramble-Pasciak CG on the saddle-point system of Eq. 2.

ORACLE (test infrastructure only).  Plain FP64 numpy on top of the MG-MG
set-up of ``oracle.ietidp.IETIDP`` (mode "mg"), written from Sec. 3.3 and
Sec. 4 of the paper and the BPCG method of Bramble and Pasciak.

The unknowns are u in V~ (torn functions whose primal values / averages are
continuous) and the multipliers lambda; Eq. 2 reads

    [ K~  B~^T ] [u     ]   [ f~ ]
    [ B~  0    ] [lambda] = [ 0  ].

Representation of V~ (Sec. 2): u = (u_Pi, w) with u_Pi the global primal
coefficients and w = (w^(k)) in ker C^(k); the function is
u^(k) = Phi^(k) A^(k) u_Pi + w^(k).  Because the primal basis Phi is
K-orthogonal to ker C (Eq. 6), K~ is block diagonal in this basis:

    K~ (u_Pi, w)   = (S_PiPi u_Pi, [P_E K^(k) w^(k)])
    B~ (u_Pi, w)   = B [Phi^(k) A^(k) u_Pi + w^(k)]
    B~^T lambda    = (sum_k A^(k)T Phi^(k)T (B^T lambda)^(k), [P_E (B^T lambda)^(k)])
    f~             = (sum_k A^(k)T Phi^(k)T f^(k), [P_E f^(k)])

with P_E the Euclidean projector on ker C^(k) (functionals on ker C are
represented by vectors in ker C).

Building blocks (Sec. 3.3, Sec. 4):
  * preconditioner for K~: the primal block exactly (Cholesky of S_PiPi); the
    Delta block by 3 V-cycles on the patch's Neumann hierarchy (K, or
    K + 1e-2 M^ on patches without a Dirichlet side), started from zero,
    wrapped in the energy-minimizing projection P = I - Phi C as in the
    local Neumann solve: Khat_Delta^{-1} g = P V3 P^T g;
  * preconditioner for the Schur complement: the scaled Dirichlet
    preconditioner M_sD^{-1} with 2 V-cycles (as in MG-MG).

Reading (the paper does not state it): BPCG needs K~ - Khat positive
definite, so each block of the preconditioner is scaled below its operator:
the primal block by omega_Pi = theta, the Delta block of patch k by
omega_k = theta (1 - rho_k^3), where rho_k estimates the energy-norm
contraction of one V-cycle (60 power iterations of I - V K on the patch's
Neumann hierarchy operator, from the fixed start vector
x_i = ((37 i) mod 101) / 101 - 1/2) and theta = 0.9.  Three V-cycles give
P V3 P^T >= (1 - rho^3) times the exact Delta inverse, so
Khat = omega (block preconditioner) stays below K~ (checked densely in the
tests; a fixed omega = 0.9 fails for p = 3 on the annulus, where
rho ~ 0.75; with p = 4, rho ~ 0.9 and 20 power iterations underestimate
it).  The iteration stops when the preconditioned residual, measured in the
BPCG inner product, has dropped by tol_outer relative to the first one; a
non-positive inner product after a step halves every scaling and restarts
from the current iterate.

BPCG with Schur preconditioner (Bramble-Pasciak transformation): with
P_BP = [Khat 0; B~ -Shat], the matrix P_BP^{-1} [K~ B~^T; B~ 0] is
self-adjoint and positive definite in the inner product
<(u,l),(v,m)> = ((K~ - Khat) u, v) + (Shat l, m); plain CG in that inner
product, where every product with K~ - Khat or Shat is formed from
quantities the iteration already has (one K~ product, one Khat^{-1}, one
Shat^{-1} per step).

Pins (tests/test_oracle_saddle.py): u equals the conforming global direct
solve; the transformed matrix is self-adjoint and the inner product
positive definite (assembled densely on a tiny problem); the iteration
counts exceed those of the dual CG of MG-MG but stay of the same order
(Tables 1-2 of the paper show 1.3-2x).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def power_start(n):
    """Fixed start vector of the contraction estimate: ((37 i) mod 101)/101 - 1/2."""
    i = np.arange(n, dtype=np.int64)
    return ((37 * i) % 101) / 101.0 - 0.5


def vcycle_contraction(mg, its=60):
    """Energy-norm contraction of one V-cycle, I - V A with A the hierarchy's
    fine operator, by power iteration (the last ratio)."""
    A = mg.A[-1]
    x = power_start(A.shape[0])
    rho = 0.0
    for _ in range(its):
        ax = A @ x
        y = x - mg.vcycle(ax)
        ex = x @ ax
        rho = np.sqrt(max(y @ (A @ y), 0.0) / ex) if ex > 0 else 0.0
        x = y / np.linalg.norm(y)
    return float(rho)


class SaddleOps:
    """The operators of Eq. 2 on V~ x Lambda for an IETIDP set up in mode "mg"."""

    def __init__(self, s, theta=0.9, ncycles=3, power_its=60, omega=None):
        if s.o.mode != "mg":
            raise ValueError("MG-MG-S needs the multigrid set-up (mode 'mg')")
        self.s = s
        self.ncycles = ncycles
        self.PE = [s._projector(k) for k in range(s.N)]
        self.rho = [vcycle_contraction(s.mgN[k], power_its) for k in range(s.N)]
        if omega is None:
            self.omega_pi = theta
            self.omega = [theta * (1.0 - r ** ncycles) for r in self.rho]
        else:                      # fixed scaling of every block (tests)
            self.omega_pi = omega
            self.omega = [omega] * s.N

    # ---- vectors on V~: (u_Pi, [w^(k)]) -------------------------------------
    def zeros_u(self):
        s = self.s
        return (np.zeros(s.nPi), [np.zeros(len(s.free[k])) for k in range(s.N)])

    @staticmethod
    def dot_u(a, b):
        return float(a[0] @ b[0] + sum(x @ y for x, y in zip(a[1], b[1])))

    @staticmethod
    def axpy_u(x, alpha, y):
        """x + alpha y"""
        return (x[0] + alpha * y[0], [a + alpha * b for a, b in zip(x[1], y[1])])

    def function(self, u):
        """Torn patch vectors u^(k) = Phi A u_Pi + w^(k)."""
        s = self.s
        out = []
        for k in range(s.N):
            v = u[1][k].copy()
            if len(s.A[k]):
                v += s.phi[k] @ u[0][s.A[k]]
            out.append(v)
        return out

    def restrict(self, g):
        """Torn functional g -> (sum_k A^T Phi^T g^(k), [P_E g^(k)])."""
        s = self.s
        gPi = np.zeros(s.nPi)
        for k in range(s.N):
            if len(s.A[k]):
                np.add.at(gPi, s.A[k], s.phi[k].T @ g[k])
        return (gPi, [self.PE[k](g[k]) for k in range(s.N)])

    # ---- operators -----------------------------------------------------------
    def K(self, u):
        s = self.s
        return (s.SPiPi @ u[0], [self.PE[k](s.K[k] @ u[1][k]) for k in range(s.N)])

    def Khat_inv(self, g):
        s = self.s
        uPi = sla.cho_solve(s.cholS, g[0]) if s.nPi else g[0].copy()
        w = []
        for k in range(s.N):
            C, phi = s.C[k], s.phi[k]
            b = g[1][k] - C.T @ (phi.T @ g[1][k]) if C.shape[0] else g[1][k].copy()
            mg = s.mgN[k]
            Af = mg.A[-1]
            z = np.zeros_like(b)
            for _ in range(self.ncycles):
                z = z + mg.vcycle(b - Af @ z)
            w.append((z - phi @ (C @ z) if C.shape[0] else z) / self.omega[k])
        return (uPi / self.omega_pi, w)

    def B(self, u):
        return self.s.Bop(self.function(u))

    def BT(self, lam):
        return self.restrict(self.s.BT(lam))

    def Shat_inv(self, r):
        return self.s.precond(r)

    def rhs(self):
        return self.restrict(self.s.f)


def bpcg(s, tol=None, maxit=None, theta=0.9, ncycles=3, power_its=60):
    """MG-MG-S solve.  Returns (u as full local tensor grids, stats dict).

    Safeguard (part of the reading): a non-positive inner product after a
    step means Khat is not below K~ (the contraction was underestimated);
    every block scaling is then halved and the iteration restarts from the
    current iterate with its residual recomputed."""
    ops = SaddleOps(s, theta, ncycles, power_its)
    tol = s.o.tol_outer if tol is None else tol
    maxit = s.o.maxit_outer if maxit is None else maxit
    f = ops.rhs()
    x_u, x_l = ops.zeros_u(), np.zeros(s.nlam)

    def start(x_u, x_l):
        # unpreconditioned residual (b - [K~ B~^T; B~ 0] x) and preconditioned r
        rt_u = ops.axpy_u(ops.axpy_u(f, -1.0, ops.K(x_u)), -1.0, ops.BT(x_l))
        rt_l = -ops.B(x_u)
        r_u = ops.Khat_inv(rt_u)
        Br = ops.B(r_u)
        r_l = ops.Shat_inv(Br - rt_l)
        return rt_u, rt_l, r_u, Br, r_l

    rt_u, rt_l, r_u, Br, r_l = start(x_u, x_l)
    rho0 = None
    it = 0
    conv = False
    restarts = 0
    p_u = p_l = Kp = KmKp = Sp = Bp = None
    rho_old = None
    hist = []
    while True:
        Kr = ops.K(r_u)
        KmKr = ops.axpy_u(Kr, -1.0, rt_u)          # (K~ - Khat) r_u
        Sr = Br - rt_l                              # Shat r_l
        rho = ops.dot_u(KmKr, r_u) + float(Sr @ r_l)
        if rho0 is None:
            rho0 = rho
        if rho < 0.0:
            if p_u is None or restarts >= 10:
                break                               # the inner product is not definite
            ops.omega_pi *= 0.5
            ops.omega = [w * 0.5 for w in ops.omega]
            rt_u, rt_l, r_u, Br, r_l = start(x_u, x_l)
            p_u = None
            restarts += 1
            continue
        hist.append(np.sqrt(rho / rho0) if rho0 > 0 else 0.0)
        if rho0 == 0.0 or rho <= tol * tol * rho0:
            conv = True
            break
        if it >= maxit:
            break
        if p_u is None:
            p_u, p_l, Kp, KmKp, Sp, Bp = r_u, r_l.copy(), Kr, KmKr, Sr.copy(), Br.copy()
        else:
            beta = rho / rho_old
            p_u = ops.axpy_u(r_u, beta, p_u)
            p_l = r_l + beta * p_l
            Kp = ops.axpy_u(Kr, beta, Kp)
            KmKp = ops.axpy_u(KmKr, beta, KmKp)
            Sp = Sr + beta * Sp
            Bp = Br + beta * Bp
        qt_u = ops.axpy_u(Kp, 1.0, ops.BT(p_l))     # K~ p_u + B~^T p_l
        qt_l = Bp                                   # B~ p_u
        q_u = ops.Khat_inv(qt_u)
        Bq = ops.B(q_u)
        q_l = ops.Shat_inv(Bq - qt_l)
        sigma = ops.dot_u(KmKp, q_u) + float(Sp @ q_l)
        if sigma <= 0.0:
            break                                   # the inner product is not definite
        alpha = rho / sigma
        x_u = ops.axpy_u(x_u, alpha, p_u)
        x_l = x_l + alpha * p_l
        rt_u = ops.axpy_u(rt_u, -alpha, qt_u)
        rt_l = rt_l - alpha * qt_l
        r_u = ops.axpy_u(r_u, -alpha, q_u)
        r_l = r_l - alpha * q_l
        Br = Br - alpha * Bq
        rho_old = rho
        it += 1
    u = s._expand(ops.function(x_u))
    return u, {"iterations": it, "converged": conv, "hist": hist, "lambda": x_l,
               "rho": ops.rho, "omega": ops.omega, "restarts": restarts}
