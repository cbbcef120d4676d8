"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point declared in include/ietidp.h (no GPU work is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ietidp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_04531_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "ietidp_solve" in names and "iga_assemble_patches" in names and "ietidp_setup" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header(lib):
    from paper_1705_04531_gb300 import ietidp
    assert set(_declared()) <= set(ietidp.EXPORTED)


def test_default_options_and_errors(lib):
    from paper_1705_04531_gb300 import ietidp
    o = ietidp.default_options()
    assert o.tol_outer == 1e-10 and o.nu_pre == 2 and o.dirichlet_vcycles == 2 and o.alpha_reg == 1e-2
    # invalid descriptor: rejected on the host before any device work
    d = ietidp.iga_domain_desc()
    d.dim = 4
    h = ctypes.c_void_p()
    rc = ietidp._lib.iga_assemble_patches(ctypes.byref(d), None, ctypes.byref(h))
    assert rc == -1 and b"dim" in ietidp._lib.ietidp_last_error()
