"""Host logic of the library on the CPU: the topology step of
iga_assemble_patches (iga_topology, no device work) against the oracle.

* counts: torn functions; conforming functions (= the oracle's global
  numbering, domain.Multipatch.nglob); classes of identified patch-boundary
  functions, shared classes and Dirichlet classes (counted from the oracle's
  local-to-global maps and its Dirichlet flags); floating patches and the
  Dirichlet side masks (the oracle's IETIDP.dmask), on 2D and 3D domains,
  uneven degrees and a domain with floating patches;
* an interface with a reversed orientation identifies the same number of
  functions (a bijection along the interface);
* invalid descriptors are rejected with IETIDP_E_INVALID_ARG: bad
  dimension, degree, box, patch index, side, a side used twice and a
  non-conforming interface.
"""
import copy

import numpy as np
import pytest

from oracle import ietidp as O
from oracle.domain import Multipatch
from paper_1705_04531_gb300 import workloads as W

DOMS = {
    "square2x2": lambda: W.square_2x2(4, 2),
    "annulus3x3": lambda: W.annulus_6x6(4, 3, grid=(3, 3)),
    "grid4x4_floating": lambda: W.uniform_grid(2, (4, 4), 2, 4, W.UNIT, None, ("vertex", "edge")),
    "uneven3x3": lambda: W.uneven_8x8(0, grid=(3, 3), nelems=(4, 8)),
    "cube2x2x2": lambda: W.cube_2x2x2(2, 2),
    "grid3x2x2": lambda: W.uniform_grid(3, (3, 2, 2), 2, 2, W.UNIT, None, ("vertex", "edge", "face")),
}


@pytest.fixture(scope="module")
def api():
    from paper_1705_04531_gb300 import build
    build.build()
    from paper_1705_04531_gb300 import ietidp
    return ietidp


def _desc(api, dom):
    d2 = copy.copy(dom)
    d2.rhs = {"kind": "none"}    # the topology does not read the load
    return api.domain_desc(d2)


def _oracle_counts(dom):
    mp = Multipatch(dom)
    copies = np.zeros(mp.nglob, dtype=np.int64)
    on_bnd = np.zeros(mp.nglob, dtype=bool)
    for k in range(dom.npatch):
        m = [n + p for n, p in zip(dom.patch_nelem(k), dom.patch_degree(k))]
        idx = np.indices(m[::-1]).reshape(len(m), -1)[::-1]    # first direction fastest
        b = np.zeros(idx.shape[1], dtype=bool)
        for r in range(len(m)):
            b |= (idx[r] == 0) | (idx[r] == m[r] - 1)
        np.add.at(copies, mp.l2g[k], 1)
        on_bnd[mp.l2g[k][b]] = True
    n_torn = int(sum(len(l) for l in mp.l2g))
    return {"n_torn": n_torn, "n_global": mp.nglob, "n_classes": int(on_bnd.sum()),
            "n_shared": int((copies >= 2).sum()), "n_dirichlet": int(mp.dirichlet.sum())}


@pytest.mark.parametrize("name", list(DOMS))
def test_topology_matches_oracle(api, name):
    dom = DOMS[name]()
    desc, keep = _desc(api, dom)
    info, dmask = api.iga_topology(desc)
    ref = _oracle_counts(dom)
    for key, v in ref.items():
        assert info[key] == v, (key, info[key], v)
    s = O.IETIDP(dom, O.Options(mode="direct"))
    assert dmask == [int(m) for m in s.dmask]
    assert info["n_floating"] == sum(s.floating)


def test_reversed_interface_identifies_as_many(api):
    dom = W.uniform_grid(2, (2, 1), 2, 4, W.UNIT, None, ("vertex",))
    desc, keep = _desc(api, dom)
    info0, _ = api.iga_topology(desc)
    desc.interfaces[0].flip[0] = 1
    info1, _ = api.iga_topology(desc)
    assert info1 == info0
    assert info0["n_global"] == info0["n_torn"] - (4 + 2)


def _expect_invalid(api, desc, word):
    with pytest.raises(api.IetidpError) as e:
        api.iga_topology(desc)
    assert api.ERRORS[e.value.code] == "INVALID_ARG"
    assert word in str(e.value), str(e.value)


def test_invalid_descriptors_rejected(api):
    def fresh():
        return _desc(api, W.uniform_grid(2, (2, 2), 2, 4, W.UNIT, None, ("vertex",)))

    desc, keep = fresh()
    desc.dim = 4
    _expect_invalid(api, desc, "dim")
    desc, keep = fresh()
    desc.patches[1].degree[0] = 0
    _expect_invalid(api, desc, "degree")
    desc, keep = fresh()
    desc.patches[2].hi[1] = desc.patches[2].lo[1]
    _expect_invalid(api, desc, "box")
    desc, keep = fresh()
    desc.interfaces[0].patch_b = 9
    _expect_invalid(api, desc, "patch index")
    desc, keep = fresh()
    desc.interfaces[0].side_a = 5
    _expect_invalid(api, desc, "side")
    desc, keep = fresh()
    desc.interfaces[1] = desc.interfaces[0]
    _expect_invalid(api, desc, "used twice")
    desc, keep = fresh()
    desc.patches[1].nelem[1] = 8        # patch 1 (right of patch 0) refined across the interface
    _expect_invalid(api, desc, "not conforming")
