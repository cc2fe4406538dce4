"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/fosb.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\**\s+\**(fosb_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fosb_mesh_create", "fosb_assemble_efie", "fosb_factor", "fosb_solve", "fosb_covariance",
              "fosb_farfield_moments"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2308_01457_gb300 import build

    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    L.fosb_version.restype = ctypes.c_char_p
    assert b"sm_103a" in L.fosb_version()


def test_invalid_arguments_rejected_on_host():
    """Argument checks happen before any device work (NULL mesh / NULL output)."""
    from paper_2308_01457_gb300 import build

    L = ctypes.CDLL(build.build())
    out = ctypes.c_void_p()
    assert L.fosb_mesh_create(None, 0, None, 0, None, ctypes.byref(out)) == 1
    assert L.fosb_assemble_efie(None, ctypes.c_double(1.0), None, 0, None, 0, None, 0, None, 0, None) == 1
    assert L.fosb_factor(None, 0, 0, 0, ctypes.byref(out), None) == 1
