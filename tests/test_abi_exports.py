"""The C-ABI library loads on a machine without a GPU and exports every
function that include/vp.h declares (no compute call is made here)."""

import ctypes
import os
import re

from paper_2203_05933_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "vp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?(vp_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vp_plan_create", "vp_eval", "vp_eval_adjoint", "vp_plan_destroy", "vp_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(build.build())
    lib.vp_status_string.restype = ctypes.c_char_p
    lib.vp_version.restype = ctypes.c_char_p
    assert lib.vp_status_string(0) == b"ok"
    assert lib.vp_status_string(1) == b"invalid argument"
    assert b"sm_103a" in lib.vp_version()
