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


def _static_fn(lib):
    fn = lib.vp_eval_direct_static
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    fn.argtypes = [I64, P, P, I32, P, I64, I64, P, P, P, P, P, I64, P]
    fn.restype = ctypes.c_int
    return fn


def test_static_entry_rejects_misaligned_points_without_gpu():
    # The pointers are never dereferenced: the argument checks run before any
    # CUDA call, so this needs no device. 0x1008 is 8-byte but not 16-byte aligned.
    lib = ctypes.CDLL(build.build())
    fn = _static_fn(lib)
    good, bad = 0x1000, 0x1008
    assert fn(10, bad, good, 1, good, 10, 10, good, None, None, None, good, 10, None) == 1
    assert fn(10, good, good, 1, good, 10, 10, bad, None, None, None, good, 10, None) == 1


def test_static_entry_rejects_correction_without_sources_without_gpu():
    lib = ctypes.CDLL(build.build())
    fn = _static_fn(lib)
    p = 0x1000
    assert fn(0, None, None, 1, None, 0, 10, p, p, p, p, p, 10, None) == 1
