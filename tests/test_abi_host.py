"""Host-side checks of the C-ABI library (no GPU): it loads, exports every symbol that
include/sap.h declares, and its host-built coupling matrices (closed forms + rotation route,
Sec. 2.1) agree with the oracle's sphere-quadrature matrices."""
import os
import re

import numpy as np
import pytest

from paper_2501_05110_gb300 import build as sap_build
from paper_2501_05110_gb300 import sapgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sap_build.build()
    return sapgpu.load_library()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "sap.h")).read()
    declared = sorted(set(re.findall(r"\b(sap_[a-z_0-9]+)\s*\(", hdr)))
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(sapgpu.EXPORTS) == declared


@pytest.mark.parametrize("lmax", [1, 3, 5, 7])
def test_library_tables_match_oracle(lib, lmax):
    from oracle import sh
    T = sh.tables(lmax)
    for a in range(3):
        np.testing.assert_allclose(sapgpu.coupling_matrix(lmax, 0, a), T["A"][a], atol=1e-12)
        np.testing.assert_allclose(sapgpu.coupling_matrix(lmax, 1, a), T["Om"][a], atol=1e-12)
        np.testing.assert_allclose(sapgpu.coupling_matrix(lmax, 4, a), T["E"][a], atol=1e-12)
        for b in range(3):
            np.testing.assert_allclose(sapgpu.coupling_matrix(lmax, 3, a, b), T["AA"][a, b], atol=1e-12)
            np.testing.assert_allclose(sapgpu.coupling_matrix(lmax, 5, a, b), T["F"][a, b], atol=1e-12)
    np.testing.assert_allclose(sapgpu.coupling_matrix(lmax, 2), T["C"], atol=1e-15)


def test_invalid_arguments_rejected(lib):
    import ctypes as C
    out = np.zeros(16)
    assert lib.sap_coupling_matrix(-1, 0, 0, 0, out.ctypes.data_as(C.POINTER(C.c_double))) == sapgpu.SAP_EINVAL
    assert lib.sap_coupling_matrix(1, 9, 0, 0, out.ctypes.data_as(C.POINTER(C.c_double))) == sapgpu.SAP_EINVAL
    h = C.c_void_p()
    d = sapgpu.Desc()
    d.ndim = 0
    assert lib.sap_create(C.byref(d), 0, C.byref(h)) == sapgpu.SAP_EINVAL
    assert b"ndim" in lib.sap_last_error(None)
