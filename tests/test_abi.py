"""The C-ABI library builds for sm_103a, loads, exports every symbol declared in
include/*.h, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

import paper_1709_10010_gb300 as pwh
from paper_1709_10010_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(pwh_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    pbuild.build()
    return pwh.lib()


def test_every_declared_symbol_is_exported_and_bound(L):
    names = declared_symbols()
    assert "pwh_apply_h" in names and "pwh_create_system" in names
    for n in names:
        assert hasattr(L, n), n
        assert n in pwh.SIGNATURES, f"{n} has no Python binding"


def test_host_side_argument_checks(L):
    h = ctypes.c_void_p()
    assert L.pwh_create_system(None, ctypes.byref(h)) == 1
    assert b"null" in L.pwh_last_error()
    d = pwh.SystemDesc()
    d.ecut_ha = -1.0
    assert L.pwh_create_system(ctypes.byref(d), ctypes.byref(h)) == 1
    assert L.pwh_apply_h(None, 1, None, 0, None, 0) == 1
    assert L.pwh_destroy_system(None) == 0
