"""The C-ABI library builds for sm_103a and exports every entry point that
include/rf.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(rf_[a-z_0-9]+)\s*\(", src))
    return names


def test_header_declares_the_boundary_entry_points():
    names = _declared()
    for n in ("rf_grid_create", "rf_assemble", "rf_gmg_setup", "rf_solve", "rf_limex_step", "rf_grid_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2506_04763_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    import paper_2506_04763_gb300 as rf
    assert _declared() == set(rf.SIGNATURES)
