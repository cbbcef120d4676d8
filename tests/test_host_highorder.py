"""CPU check of the library's host builder of the high-order multigrid (Sec. 4,
p >= 4): the 1D generalized eigenbases and scalings of the subspace-corrected
mass smoother and the L2-projection prolongations, built in FP64 C++ with no
device work (ietidp_ho_patch_operators), against the oracle's
(oracle/highorder.py, LAPACK).

The two sides' eigenvector bases may differ inside clusters of close
eigenvalues; the smoother's operator L^-1 = U diag(Dinv) U^T and the
prolongation do not, so these are compared (relative 1e-10; both are FP64
computations of the same well-conditioned quantities: measured 3e-13).
Patches: curved (quarter annulus) with and without a Dirichlet side and a
floating one (regularised), degrees 5 and 7, and a 3D box."""
import numpy as np
import pytest

from oracle import assembly, highorder as H
from oracle import ietidp as O
from paper_1705_04531_gb300 import workloads as W


@pytest.fixture(scope="module")
def api():
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp
    return ietidp


def _uneven():
    return W.Domain(2, (2, 2), [[5, 7], [7, 5]], [[8, 8], [8, 16]], W.UNIT, {"kind": "sin2d"},
                    (W.PRIMAL_VERTEX, W.PRIMAL_EDGE), "uneven_ho")


CASES = [
    ("annulus6x6_p4", lambda: W.annulus_6x6(16, 4), (0, 7, 35)),
    ("square_p5", lambda: W.uniform_grid(2, (2, 2), 5, 8), (0,)),
    ("uneven_p5_p7", _uneven, (1, 3)),
    ("cube_p4", lambda: W.cube_2x2x2(4, 4), (0, 7)),
]


def _kron_all(mats):
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(m, out)      # first direction fastest
    return out


@pytest.mark.parametrize("name,make,patches", CASES)
def test_host_builder_matches_oracle(api, name, make, patches):
    dom = make()
    orc = O.IETIDP(dom, O.Options(mode="direct"))
    allsides = (1 << (2 * dom.dim)) - 1
    alpha = 1e-2
    for k in patches:
        K, _, _ = assembly.assemble_patch(dom, k, with_rhs=False)
        for kind, mask in ((0, orc.dmask[k]), (1, allsides)):
            al = alpha if (kind == 0 and orc.dmask[k] == 0) else 0.0
            mg = H.HighOrderMG(dom, k, K, mask, al)
            Us, Ps, Dinv = api.ho_patch_operators(dom, k, kind, alpha)
            U = _kron_all(Us)
            Linv = U @ np.diag(Dinv) @ U.T
            n = Linv.shape[0]
            assert n == len(mg.free)
            ref = np.array([mg.smooth_inv(e) for e in np.eye(n)]).T
            err = np.abs(Linv - ref).max() / np.abs(ref).max()
            assert err <= 1e-10, (name, k, kind, err)
            Pm = _kron_all(Ps)
            Pref = mg.P.toarray()
            errp = np.abs(Pm - Pref).max() / np.abs(Pref).max()
            assert errp <= 1e-10, (name, k, kind, errp)


def test_host_builder_rejects_bad_arguments(api):
    dom = W.uniform_grid(2, (2, 2), 4, 8)
    with pytest.raises(api.IetidpError):
        api.ho_patch_operators(dom, 0, 2)
    bad = W.uniform_grid(2, (2, 2), 8, 8)
    with pytest.raises(api.IetidpError):
        api.ho_patch_operators(bad, 0, 0)
