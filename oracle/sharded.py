"""Patch-sharded dual PCG: the exchange step of a multi-GPU IETI-DP solve,
with ranks as processes.

ORACLE (test infrastructure only).  Plain FP64 numpy on top of a fully set-up
``oracle.ietidp.IETIDP`` (every rank sets up the whole problem; only the
per-iteration work is sharded).

Sec. 2: K~^{-1} is block diagonal in the patches apart from the primal
(coarse) part, and the scaled Dirichlet preconditioner is a sum of
independent patch contributions, so the local problems of an outer iteration
shard by patch.  Each rank owns a contiguous block of patches and keeps the
multiplier-space vectors (lambda, r, p, z, q) whole on every rank.  What the
ranks exchange, per outer iteration, is three sums (all-reduce):

  F p      r_Pi = sum_k A_k^T Phi_k^T (B_k^T p)       n_Pi values
           B K~^{-1} B^T p, partial per rank          n_lambda values
  M^{-1} r B_D S B_D^T r, partial per rank            n_lambda values

plus the primal coarse solve, replicated (S_PiPi is small, Sec. 3.3).  Dot
products act on the replicated vectors and need no exchange.  A multiplier
couples two torn copies of one dof; its row of B takes the +1 copy from the
rank owning the first patch and the -1 copy from the rank owning the second,
so the partial sums add up to B u exactly as one process forms it.

``allreduce(x)`` returns the elementwise sum of x over the ranks (a numpy
array of the same shape); the test passes one built on torch.distributed
(gloo).  ``counts`` records the exchanges (calls and values).

Pins (tests/test_oracle_sharded.py): with 2 ranks the solution equals the
single-process oracle's to 1e-12 and the outer iteration count agrees; the
exchanged values per outer iteration are n_Pi + 2 n_lambda; with one rank the
arithmetic is the single-process one.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .ietidp import IETIDP, lanczos_kappa


def owned(N, rank, world):
    """Contiguous block of patches of a rank."""
    return range(rank * N // world, (rank + 1) * N // world)


class Sharded:
    def __init__(self, s: IETIDP, rank, world, allreduce):
        self.s = s
        self.own = owned(s.N, rank, world)
        self.mine = np.zeros(s.N, dtype=bool)
        self.mine[list(self.own)] = True
        self._ar = allreduce
        self.counts = {"calls": 0, "values": 0}

    def allreduce(self, x):
        x = np.asarray(x, dtype=np.float64)
        self.counts["calls"] += 1
        self.counts["values"] += x.size
        return self._ar(x)

    def BT(self, lam_vec, scaled=False):
        """B_k^T lambda on the owned patches (None elsewhere)."""
        s = self.s
        out = [np.zeros(len(s.free[k])) if self.mine[k] else None for k in range(s.N)]
        for i, (ka, la, kb, lb) in enumerate(s.lam):
            if self.mine[ka]:
                out[ka][la] += (1.0 / s.mult[ka][la] if scaled else 1.0) * lam_vec[i]
            if self.mine[kb]:
                out[kb][lb] -= (1.0 / s.mult[kb][lb] if scaled else 1.0) * lam_vec[i]
        return out

    def B_partial(self, u, scaled=False):
        """This rank's share of B u (its copies' terms of every multiplier)."""
        s = self.s
        q = np.zeros(s.nlam)
        for i, (ka, la, kb, lb) in enumerate(s.lam):
            if self.mine[ka]:
                q[i] += (1.0 / s.mult[ka][la] if scaled else 1.0) * u[ka][la]
            if self.mine[kb]:
                q[i] -= (1.0 / s.mult[kb][lb] if scaled else 1.0) * u[kb][lb]
        return q

    def Ktilde_inv(self, g):
        """K~^{-1} g on the owned patches: primal part from the all-reduced
        r_Pi and the replicated coarse solve, Delta part per owned patch."""
        s = self.s
        rPi = np.zeros(s.nPi)
        for k in self.own:
            if len(s.A[k]):
                np.add.at(rPi, s.A[k], s.phi[k].T @ g[k])
        if s.nPi:
            rPi = self.allreduce(rPi)
        uPi = sla.cho_solve(s.cholS, rPi) if s.nPi else rPi
        out = [None] * s.N
        for k in self.own:
            u = s.delta_solve(k, g[k])
            if len(s.A[k]):
                u = u + s.phi[k] @ uPi[s.A[k]]
            out[k] = u
        return out

    def F(self, lam):
        return self.allreduce(self.B_partial(self.Ktilde_inv(self.BT(lam))))

    def precond(self, r):
        v = self.BT(r, scaled=True)
        w = [self.s.schur_apply(k, v[k]) if self.mine[k] else None for k in range(self.s.N)]
        return self.allreduce(self.B_partial(w, scaled=True))

    def jump_scale(self, u):
        s = self.s
        t = 0.0
        for (ka, la, kb, lb) in s.lam:
            if self.mine[ka]:
                t += u[ka][la] ** 2
            if self.mine[kb]:
                t += u[kb][lb] ** 2
        return float(np.sqrt(self.allreduce(np.array([t]))[0]))

    def solve(self):
        """The outer PCG of oracle.ietidp.IETIDP.solve with sharded operators.
        Returns (owned patches' full local solutions as {k: vector}, stats)."""
        s = self.s
        o = s.o
        st = {"outer_it": 0, "converged": False, "alphas": [], "betas": []}
        fr = s.f
        u0 = self.Ktilde_inv(fr)
        if s.nlam == 0:
            st["converged"] = True
            return self._expand(u0), st
        d = self.allreduce(self.B_partial(u0))
        lam = np.zeros(s.nlam)
        r = d.copy()
        nd = np.linalg.norm(d)
        if nd <= o.tol_outer * self.jump_scale(u0):
            st["converged"] = True
        else:
            z = self.precond(r)
            p = z.copy()
            rz = r @ z
            for it in range(1, o.maxit_outer + 1):
                q = self.F(p)
                alpha = rz / (p @ q)
                lam += alpha * p
                r -= alpha * q
                st["alphas"].append(alpha)
                st["outer_it"] = it
                if np.linalg.norm(r) / nd <= o.tol_outer:
                    st["converged"] = True
                    break
                z = self.precond(r)
                rz_new = r @ z
                beta = rz_new / rz
                st["betas"].append(beta)
                rz = rz_new
                p = z + beta * p
        st["kappa"] = lanczos_kappa(st["alphas"], st["betas"])
        bt = self.BT(lam)
        u = self.Ktilde_inv([fr[k] - bt[k] if self.mine[k] else None for k in range(s.N)])
        return self._expand(u), st

    def _expand(self, u):
        s = self.s
        out = {}
        for k in self.own:
            full = np.zeros(int(np.prod(s.m[k])))
            full[s.free[k]] = u[k]
            out[k] = full
        return out
