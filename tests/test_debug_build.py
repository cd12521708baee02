"""The bounds-checked debug build compiles for sm_103a and exports the fault
word of every checked translation unit; the product library exports none of
them (its checks compile away).  No GPU is needed: nvcc cross-compiles."""
import ctypes
import os

import pytest

UNITS = ("sort", "build", "upward", "walk", "periodic", "adjoint")


@pytest.mark.timeout(900)
def test_debug_library_exports_fault_words():
    from paper_1407_2600_gb300 import build as libbuild
    dbg = libbuild.build(debug_bounds=True)
    assert os.path.basename(dbg) == "libnbody_dbg.so"
    L = ctypes.CDLL(dbg)
    for u in UNITS:
        assert hasattr(L, "nbody_dbg_fault_" + u), u
    prod = ctypes.CDLL(libbuild.build())
    for u in UNITS:
        assert not hasattr(prod, "nbody_dbg_fault_" + u), u
