"""Pins of the Schoeberl-Zulehner CG for the primal basis (oracle/szcg.py).

* the SZ basis equals the direct solution of Eq. 6 (saddle LU of the D-D
  oracle) and satisfies C phi = I and phi^T K v = 0 on ker C;
* dense, on a tiny patch: Khat - K is positive definite (the SZ condition,
  with Khat^{-1} = 0.99 V), the SZ preconditioner inverts P exactly, and the
  preconditioned saddle matrix is self-adjoint in the D inner product;
* SZ-CG needs fewer iterations than the null-space CG of R10.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ietidp as O
from oracle import szcg
from paper_1705_04531_gb300 import workloads as W

DOMS = {
    "annulus3x3": lambda: W.annulus_6x6(8, 3, grid=(3, 3)),
    "grid3_floating": lambda: W.uniform_grid(2, (3, 3), 2, 8, W.UNIT, None, ("vertex", "edge")),
    "cube": lambda: W.cube_2x2x2(4, 2),
    "uneven3x3": lambda: W.uneven_8x8(0, grid=(3, 3), nelems=(8, 16, 32)),
}


@pytest.mark.parametrize("name", list(DOMS))
def test_sz_basis_equals_direct(name):
    dom = DOMS[name]()
    sd = O.IETIDP(dom, O.Options(mode="direct"))
    sm = O.IETIDP(dom, O.Options(mode="mg"))
    phis, its = szcg.sz_basis(sm)
    for k in range(sd.N):
        if sd.C[k].shape[0] == 0:
            continue
        ref = sd.phi[k]
        assert np.abs(phis[k] - ref).max() <= 1e-8 * max(1.0, np.abs(ref).max()), k
        C = sd.C[k].toarray()
        assert np.abs(C @ phis[k] - np.eye(C.shape[0])).max() < 1e-9
        Z = sla.null_space(C)
        KZ = sd.K[k] @ Z
        assert np.abs(phis[k].T @ KZ).max() <= 1e-8 * np.abs(KZ).max()
    # fewer iterations than the null-space CG of the MG-MG set-up
    assert np.mean(its) < np.mean(sm.stats.basis_its), (np.mean(its), np.mean(sm.stats.basis_its))


def test_sz_conditions_dense_tiny():
    dom = W.uniform_grid(2, (3, 3), 2, 8, W.UNIT, None, ("vertex", "edge"))
    s = O.IETIDP(dom, O.Options(mode="mg"))
    for k in (0, 4):                     # a corner patch and the floating centre patch
        pz = szcg.SZPatch(s, k)
        n, npi = pz.W.shape
        K = pz.K.toarray()
        Khi = np.column_stack([pz.khat_inv(e) for e in np.eye(n)])
        assert np.abs(Khi - Khi.T).max() < 1e-10 * np.abs(Khi).max()
        Khat = np.linalg.inv(0.5 * (Khi + Khi.T))
        assert np.linalg.eigvalsh(Khat - K).min() > 0          # Khat > K
        D2 = pz.C @ Khi @ pz.C.T - szcg.HHAT_SCALE * pz.H
        assert np.linalg.eigvalsh(0.5 * (D2 + D2.T)).min() > 0  # Hhat < C Khat^{-1} C^T
        # the preconditioner application inverts P
        P = np.block([[Khat, pz.C.T], [pz.C, pz.C @ Khi @ pz.C.T - szcg.HHAT_SCALE * pz.H]])
        A = np.block([[K, pz.C.T], [pz.C, np.zeros((npi, npi))]])
        rng = np.random.default_rng(k)
        r1, r2 = rng.standard_normal(n), rng.standard_normal(npi)
        z1, z2 = pz.precond(r1, r2)
        back = P @ np.concatenate([z1, z2])
        assert np.abs(back - np.concatenate([r1, r2])).max() < 1e-8 * np.abs(back).max()
        # P^{-1} A is self-adjoint and positive definite in the D = P - A inner product
        Dm = P - A
        M = np.linalg.solve(P, A)
        DM = Dm @ M
        assert np.abs(DM - DM.T).max() < 1e-8 * np.abs(DM).max()
        assert np.linalg.eigvalsh(0.5 * (Dm + Dm.T)).min() > 0
        assert np.linalg.eigvalsh(0.5 * (DM + DM.T)).min() > 0
