"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/nrs.h declares.  No compute call is made here."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "nrs.h")).read()
    return sorted(set(re.findall(r"^\w[\w\s\*]*?\b(nrs_\w+)\s*\(", hdr, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("nrs_create", "nrs_destroy", "nrs_nearest_build", "nrs_assemble", "nrs_factor",
                 "nrs_solve", "nrs_step"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2001_06468_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2001_06468_gb300 import build as B
    B.build()
    from paper_2001_06468_gb300 import nrs
    assert sorted(nrs.EXPORTS) == _declared()
