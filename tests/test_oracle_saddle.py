"""Pins of the MG-MG-S oracle (BPCG on the saddle-point system, Eq. 2).

* the solution equals the conforming global direct solve (the definition);
* on a tiny problem, assembled densely in a basis of V~: the preconditioner
  Khat^{-1} is symmetric, K~ - Khat is positive definite (the BPCG condition,
  which the contraction-based scaling guarantees and omega = 1 violates), K~ is the block-diagonal operator of
  the energy-minimizing basis (its primal block equals S_PiPi and is
  K-orthogonal to the Delta block), B~ and B~^T are adjoint, and the Schur
  preconditioner is symmetric positive semidefinite;
* outer iteration counts exceed those of the dual CG of MG-MG by a moderate
  factor (the paper's tables: 1.3-2x).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ietidp as O
from oracle import saddle
from oracle.domain import Multipatch
from paper_1705_04531_gb300 import workloads as W


def relerr(got, ref):
    return np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(got, ref)) / sum(np.sum(b ** 2) for b in ref))


DOMS = {
    "square": lambda: W.random_quad_rhs(W.square_2x2(8, 2), seed=21),
    "annulus3x3": lambda: W.annulus_6x6(8, 3, grid=(3, 3)),
    "grid3_floating": lambda: W.random_quad_rhs(W.uniform_grid(2, (3, 3), 2, 8, W.UNIT, None,
                                                               ("vertex", "edge")), seed=22),
    "cube": lambda: W.random_quad_rhs(W.cube_2x2x2(4, 2), seed=23),
    "uneven3x3": lambda: W.random_quad_rhs(W.uneven_8x8(0, grid=(3, 3), nelems=(8, 16, 32)), seed=32),
}


@pytest.mark.parametrize("name", list(DOMS))
def test_bpcg_matches_direct(name):
    dom = DOMS[name]()
    mp = Multipatch(dom)
    ref = mp.to_patches(mp.solve_global())
    s = O.IETIDP(dom, O.Options(mode="mg"))
    u, st = saddle.bpcg(s)
    assert st["converged"], st["iterations"]
    assert relerr(u, ref) <= 1e-8, relerr(u, ref)
    # continuity of the torn solution
    assert np.linalg.norm(s.jump(u)) <= 1e-8 * np.sqrt(sum(np.sum(x ** 2) for x in u))


def _dense(ops, s):
    """Dense matrices of the saddle operators in an orthonormal basis of V~."""
    Z = [sla.null_space(s.C[k].toarray()) if s.C[k].shape[0] else np.eye(len(s.free[k]))
         for k in range(s.N)]
    dims = [s.nPi] + [z.shape[1] for z in Z]
    off = np.concatenate([[0], np.cumsum(dims)])
    n = int(off[-1])

    def to_u(c):
        return (c[:s.nPi].copy(), [Z[k] @ c[off[k + 1]:off[k + 2]] for k in range(s.N)])

    def from_u(u):
        return np.concatenate([u[0]] + [Z[k].T @ u[1][k] for k in range(s.N)])

    E = np.eye(n)
    Kt = np.column_stack([from_u(ops.K(to_u(E[:, j]))) for j in range(n)])
    Khi = np.column_stack([from_u(ops.Khat_inv(to_u(E[:, j]))) for j in range(n)])
    Bt = np.column_stack([ops.B(to_u(E[:, j])) for j in range(n)])
    BTm = np.column_stack([from_u(ops.BT(e)) for e in np.eye(s.nlam)])
    Si = np.column_stack([ops.Shat_inv(e) for e in np.eye(s.nlam)])
    return Kt, Khi, Bt, BTm, Si, Z


def test_saddle_operators_dense_tiny():
    dom = W.random_quad_rhs(W.uniform_grid(2, (2, 2), 2, 8, W.UNIT, None, ("vertex", "edge")), seed=24)
    s = O.IETIDP(dom, O.Options(mode="mg"))
    ops = saddle.SaddleOps(s)
    Kt, Khi, Bt, BTm, Si, Z = _dense(ops, s)
    sym = lambda M: np.abs(M - M.T).max() / np.abs(M).max()
    assert sym(Kt) < 1e-12
    assert sym(Khi) < 1e-10
    assert sym(Si) < 1e-10
    # primal block of K~ is S_PiPi, off-diagonal blocks vanish (Eq. 6)
    npi = s.nPi
    assert np.abs(Kt[:npi, :npi] - s.SPiPi).max() < 1e-10 * np.abs(s.SPiPi).max()
    assert np.abs(Kt[:npi, npi:]).max() < 1e-10 * np.abs(Kt).max()
    # K~ positive definite, K~ - Khat positive definite (BPCG condition)
    assert np.linalg.eigvalsh(Kt).min() > 0
    Khat = np.linalg.inv(Khi)
    ev = np.linalg.eigvalsh(0.5 * (Kt - Khat + (Kt - Khat).T))
    assert ev.min() > 0, ev.min()
    # without the scaling (omega = 1) the condition fails: the reading matters
    ops1 = saddle.SaddleOps(s, omega=1.0)
    _, Khi1, _, _, _, _ = _dense(ops1, s)
    ev1 = np.linalg.eigvalsh(Kt - np.linalg.inv(0.5 * (Khi1 + Khi1.T)))
    assert ev1.min() < 1e-6 * np.abs(Kt).max()
    # B~ and B~^T are adjoint; Shat^{-1} positive semidefinite
    assert np.abs(Bt.T - BTm).max() < 1e-12 * max(1.0, np.abs(Bt).max())
    assert np.linalg.eigvalsh(0.5 * (Si + Si.T)).min() > -1e-12 * np.abs(Si).max()
    # the saddle system in this basis has the conforming solution
    f = ops.rhs()
    fc = np.concatenate([f[0]] + [Z[k].T @ f[1][k] for k in range(s.N)])
    M = np.block([[Kt, Bt.T], [Bt, np.zeros((s.nlam, s.nlam))]])
    sol = np.linalg.lstsq(M, np.concatenate([fc, np.zeros(s.nlam)]), rcond=None)[0]
    uc = sol[:Kt.shape[0]]
    dims = np.concatenate([[0], np.cumsum([s.nPi] + [z.shape[1] for z in Z])])
    u = (uc[:s.nPi], [Z[k] @ uc[dims[k + 1]:dims[k + 2]] for k in range(s.N)])
    mp = Multipatch(dom)
    ref = mp.to_patches(mp.solve_global())
    assert relerr(s._expand(ops.function(u)), ref) < 1e-9


def test_contraction_estimate_bounds_block_condition():
    """Per patch, omega_k P V3 P^T^{-1} < K on ker C: checked densely, and the
    estimate agrees with the exact spectral radius of the V-cycle error
    propagation (dense eigenvalues)."""
    dom = W.annulus_6x6(8, 3, grid=(2, 2))
    s = O.IETIDP(dom, O.Options(mode="mg"))
    for k in range(s.N):
        mg = s.mgN[k]
        A = mg.A[-1].toarray()
        n = A.shape[0]
        V = np.column_stack([mg.vcycle(e) for e in np.eye(n)])
        E = np.eye(n) - V @ A
        Lc = np.linalg.cholesky(A)
        rho_exact = np.abs(np.linalg.eigvals(Lc.T @ E @ np.linalg.inv(Lc.T))).max()
        rho_est = saddle.vcycle_contraction(mg)
        assert rho_est <= rho_exact * (1 + 1e-6)
        assert rho_est >= 0.98 * rho_exact, (rho_est, rho_exact)


def test_bpcg_iterations_exceed_dual_cg_moderately():
    dom = DOMS["annulus3x3"]()
    s = O.IETIDP(dom, O.Options(mode="mg"))
    s.solve()
    its_cg = s.stats.outer_it
    _, st = saddle.bpcg(s)
    assert its_cg <= st["iterations"] <= 4 * its_cg, (its_cg, st["iterations"])
