"""Plain CPU FP64 oracle for the volume-potential hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``, never by the library. It shares no
code with the CUDA path. The arithmetic lives in ``vp_oracle.c`` (plain C,
OpenMP over targets, Neumaier-compensated FP64 sums); this module only builds
it with gcc and marshals numpy arrays.

Definitions (arXiv 2203.05933):
  * ``evaluate``  V_i = sum_{r_j != t_i} w_j f_j G(r_j, t_i) + (Pi f)_i, with
                  G = -(1/2pi) log|r - r0| (Sec. 2.1), the smooth rule of
                  Eq. Tk_smooth_quad with Jacobians folded into w, and the sparse
                  correction matrix Pi of Sec. 4 (paragraph after Eq. nsrcs).
  * ``adjoint``   (A^T g)_j = w_j sum_i G(r_j, t_i) g_i + (Pi^T g)_j.
  * ``grad_targets`` dL/dt_i for upstream gradient g = dL/dV, Pi held fixed.

A coincident (bitwise equal) source/target pair contributes nothing.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libvp_oracle.so")
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.vpo_eval.argtypes = [_i64, _ptr, _ptr, _i32, _ptr, _i64, _i64, _ptr,
                                 _ptr, _ptr, _ptr, _ptr, _i64, ctypes.c_int]
        lib.vpo_adjoint.argtypes = lib.vpo_eval.argtypes
        lib.vpo_grad_targets.argtypes = [_i64, _ptr, _ptr, _i32, _ptr, _i64, _ptr, _i64,
                                         _i64, _ptr, _ptr, ctypes.c_int]
        lib.vpo_grad_scale.argtypes = lib.vpo_grad_targets.argtypes
        lib.vpo_max_threads.argtypes = []
        for fn in (lib.vpo_eval, lib.vpo_adjoint, lib.vpo_grad_targets, lib.vpo_grad_scale, lib.vpo_max_threads):
            fn.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().vpo_max_threads())


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(csr, n_rows):
    if csr is None:
        return None, None, None
    rowptr, col, val = csr
    rowptr = _c(rowptr, np.int64)
    col = _c(col, np.int32)
    val = _c(val, np.float64)
    if rowptr.shape != (n_rows + 1,) or col.shape != val.shape or rowptr[-1] != col.size:
        raise ValueError("malformed CSR")
    return rowptr, col, val


def _dens(f, n):
    f = _c(f, np.float64)
    if f.ndim == 1:
        f = f[None, :]
    if f.shape[1] != n:
        raise ValueError("density length mismatch")
    return f


def evaluate(src_xy, w, f, tgt_xy, csr=None, nthreads: int = 0) -> np.ndarray:
    """V[d, i] for densities f[d, j] (1-D f gives a 1-D result)."""
    squeeze = np.ndim(f) == 1
    src_xy = _c(src_xy, np.float64).reshape(-1, 2)
    tgt_xy = _c(tgt_xy, np.float64).reshape(-1, 2)
    w = _c(w, np.float64)
    f = _dens(f, src_xy.shape[0])
    rowptr, col, val = _csr(csr, tgt_xy.shape[0])
    out = np.empty((f.shape[0], tgt_xy.shape[0]), np.float64)
    rc = _load().vpo_eval(src_xy.shape[0], _p(src_xy), _p(w), f.shape[0], _p(f), f.shape[1],
                          tgt_xy.shape[0], _p(tgt_xy), _p(rowptr), _p(col), _p(val),
                          _p(out), out.shape[1], int(nthreads))
    if rc != 0:
        raise RuntimeError(f"vpo_eval failed ({rc})")
    return out[0] if squeeze else out


def adjoint(src_xy, w, g, tgt_xy, csr=None, nthreads: int = 0) -> np.ndarray:
    """(A^T g)[d, j] for upstream values g[d, i] at the targets."""
    squeeze = np.ndim(g) == 1
    src_xy = _c(src_xy, np.float64).reshape(-1, 2)
    tgt_xy = _c(tgt_xy, np.float64).reshape(-1, 2)
    w = _c(w, np.float64)
    g = _dens(g, tgt_xy.shape[0])
    rowptr, col, val = _csr(csr, tgt_xy.shape[0])
    out = np.empty((g.shape[0], src_xy.shape[0]), np.float64)
    rc = _load().vpo_adjoint(src_xy.shape[0], _p(src_xy), _p(w), g.shape[0], _p(g), g.shape[1],
                             tgt_xy.shape[0], _p(tgt_xy), _p(rowptr), _p(col), _p(val),
                             _p(out), out.shape[1], int(nthreads))
    if rc != 0:
        raise RuntimeError(f"vpo_adjoint failed ({rc})")
    return out[0] if squeeze else out


def grad_targets(src_xy, w, f, g, tgt_xy, nthreads: int = 0) -> np.ndarray:
    """dL/dt[i, 2] = sum_d g[d, i] dV[d, i]/dt_i with the correction held fixed."""
    src_xy = _c(src_xy, np.float64).reshape(-1, 2)
    tgt_xy = _c(tgt_xy, np.float64).reshape(-1, 2)
    w = _c(w, np.float64)
    f = _dens(f, src_xy.shape[0])
    g = _dens(g, tgt_xy.shape[0])
    if g.shape[0] != f.shape[0]:
        raise ValueError("f and g must hold the same number of densities")
    out = np.empty((tgt_xy.shape[0], 2), np.float64)
    rc = _load().vpo_grad_targets(src_xy.shape[0], _p(src_xy), _p(w), f.shape[0], _p(f), f.shape[1],
                                  _p(g), g.shape[1], tgt_xy.shape[0], _p(tgt_xy), _p(out),
                                  int(nthreads))
    if rc != 0:
        raise RuntimeError(f"vpo_grad_targets failed ({rc})")
    return out


def grad_scale(src_xy, w, f, g, tgt_xy, nthreads: int = 0) -> np.ndarray:
    """Per-target normaliser of dL/dt errors: sum_d |g[d, i]| sum_j |w_j f[d, j]| / (2 pi |t_i - r_j|)
    (coincident pairs skipped), the sum of the absolute values of the gradient's terms."""
    src_xy = _c(src_xy, np.float64).reshape(-1, 2)
    tgt_xy = _c(tgt_xy, np.float64).reshape(-1, 2)
    w = _c(w, np.float64)
    f = _dens(f, src_xy.shape[0])
    g = _dens(g, tgt_xy.shape[0])
    if g.shape[0] != f.shape[0]:
        raise ValueError("f and g must hold the same number of densities")
    out = np.empty(tgt_xy.shape[0], np.float64)
    rc = _load().vpo_grad_scale(src_xy.shape[0], _p(src_xy), _p(w), f.shape[0], _p(f), f.shape[1],
                                _p(g), g.shape[1], tgt_xy.shape[0], _p(tgt_xy), _p(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"vpo_grad_scale failed ({rc})")
    return out


def csr_rows(csr, rows):
    """Sub-CSR holding only the given rows (for target subsamples)."""
    rowptr, col, val = csr
    rowptr = np.asarray(rowptr, np.int64)
    rows = np.asarray(rows, np.int64)
    lens = rowptr[rows + 1] - rowptr[rows]
    new_ptr = np.zeros(rows.size + 1, np.int64)
    np.cumsum(lens, out=new_ptr[1:])
    idx = np.concatenate([np.arange(rowptr[r], rowptr[r + 1]) for r in rows]) if rows.size else \
        np.zeros(0, np.int64)
    return new_ptr, np.asarray(col)[idx], np.asarray(val)[idx]
