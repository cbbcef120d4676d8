"""Pins of the conforming global solve (the definition of the method's
result, Eq. 1 on the multipatch space of Sec. 2) and of the multigrid
oracle (Sec. 4)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assembly, multigrid
from oracle.domain import Multipatch
from paper_1705_04531_gb300 import workloads as W


def _rates(doms):
    errs = [Multipatch(d).l2_error(Multipatch(d).solve_global()) for d in doms]
    return np.log2(np.array(errs[:-1]) / np.array(errs[1:])), errs


def test_l2_rate_square_p2():
    rates, _ = _rates([W.square_2x2(n, 2) for n in (4, 8, 16)])
    assert rates[-1] > 2.8          # order p + 1 = 3


def test_l2_rate_annulus_p3():
    rates, _ = _rates([W.annulus_6x6(n, 3, grid=(2, 2)) for n in (2, 4, 8)])
    assert rates[-1] > 3.6          # order p + 1 = 4


def test_l2_rate_cube_p2():
    rates, _ = _rates([W.cube_2x2x2(n, 2) for n in (2, 4)])
    assert rates[-1] > 2.6


def test_single_patch_reduces_to_galerkin():
    dom = W.uniform_grid(2, (1, 1), 2, 8)
    mp = Multipatch(dom)
    u = mp.solve_global()
    K, f, _ = assembly.assemble_patch(dom, 0)
    fr = np.nonzero(multigrid.free_mask((10, 10), 0b1111))[0]
    ref = spla.spsolve(K[fr][:, fr].tocsc(), f[fr])
    assert np.allclose(u[fr], ref, atol=1e-13)


def _mg(n=16, p=2, mask=0b1111, alpha=0.0):
    dom = W.square_2x2(n, p)
    K, _, _ = assembly.assemble_patch(dom, 0)
    h = multigrid.Hierarchy(K, (n, n), (p, p))
    return multigrid.MGOperator(h, mask, alpha)


def _vmatrix(mg):
    n = mg.A[-1].shape[0]
    return np.array([mg.vcycle(e) for e in np.eye(n)]).T


def test_vcycle_symmetric_and_contracting():
    for n in (8, 16):
        mg = _mg(n)
        V = _vmatrix(mg)
        assert np.abs(V - V.T).max() < 1e-12 * np.abs(V).max()
        E = np.eye(V.shape[0]) - V @ mg.A[-1].toarray()
        rho = np.max(np.abs(np.linalg.eigvals(E)))
        assert rho < 0.3, rho


def test_vcycle_one_level_is_exact():
    mg = _mg(4)
    assert mg.h.L == 1
    b = np.random.default_rng(0).standard_normal(mg.A[0].shape[0])
    assert np.allclose(mg.A[0] @ mg.vcycle(b), b, atol=1e-12)


def test_colors_decouple():
    mg = _mg(8, 3)
    A = mg.A[-1]
    assert len(mg.colors[-1]) == 16
    for idx, _, _ in mg.colors[-1]:
        sub = A[idx][:, idx].toarray()
        assert np.count_nonzero(sub - np.diag(np.diag(sub))) == 0


def test_regularized_floating_pcg():
    mg = _mg(16, 2, mask=0, alpha=1e-2)
    K = mg.h.K[-1]
    b = np.random.default_rng(1).standard_normal(K.shape[0])
    b -= b.mean()                          # consistent: K 1 = 0
    x, it, ok = multigrid.pcg(lambda v: K @ v, b, mg.vcycle, 1e-12)
    assert ok and it < 40
    assert np.linalg.norm(K @ x - b) <= 1e-11 * np.linalg.norm(b)


def test_pcg_matches_direct():
    mg = _mg(16, 2)
    A = mg.A[-1]
    b = np.random.default_rng(2).standard_normal(A.shape[0])
    x, it, ok = multigrid.pcg(lambda v: A @ v, b, mg.vcycle, 1e-12)
    assert ok
    assert np.allclose(x, spla.spsolve(A.tocsc(), b), atol=1e-11)
