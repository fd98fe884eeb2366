"""Plain CPU FP64 oracle for the modified-Helmholtz volume potential.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU legs of ``bench.py``, never by the library. It shares no code
with the CUDA path.

Definition (arXiv 2203.05933, Sec. 2: the Green function of L = -Delta + lambda^2,
used for the volume potential exactly as the Laplace one, Sec. 5):

    V_i = sum_{r_j != t_i} w_j f_j G(r_j, t_i) + (Pi f)_i,
    G(r, r0) = (lambda^2 / 2 pi) K0(lambda |r - r0|),

with the smooth rule of Eq. Tk_smooth_quad (Jacobians folded into w) and the
sparse correction matrix Pi of Sec. 4. A coincident (bitwise equal) pair
contributes nothing. K0 is ``scipy.special.k0`` and the CSR product
``scipy.sparse`` (library primitives); each target's sum over the sources is
numpy's pairwise sum. The adjoint is (A^T g)_j = w_j sum_i G(r_j, t_i) g_i +
(Pi^T g)_j (G is symmetric).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse
from scipy.special import k0

_CHUNK_PAIRS = 1 << 22


def _kernel_block(src, tgt, lam):
    """G(r_j, t_i) for a block of targets, zero for coincident pairs."""
    dx = tgt[:, 0][:, None] - src[:, 0][None, :]
    dy = tgt[:, 1][:, None] - src[:, 1][None, :]
    r = np.hypot(dx, dy)
    g = np.zeros_like(r)
    nz = r > 0.0
    g[nz] = (lam * lam / (2.0 * math.pi)) * k0(lam * r[nz])
    return g


def _dens(f, n):
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 1:
        f = f[None, :]
    if f.shape[1] != n:
        raise ValueError("density length does not match")
    return f


def _csr_matrix(csr, n_rows, n_cols):
    rowptr, col, val = csr
    return scipy.sparse.csr_matrix((np.asarray(val, np.float64), np.asarray(col, np.int64),
                                    np.asarray(rowptr, np.int64)), shape=(n_rows, n_cols))


def evaluate(src_xy, w, f, tgt_xy, lam: float, csr=None) -> np.ndarray:
    """V [ndens, n_tgt] (see the module docstring)."""
    src = np.asarray(src_xy, np.float64).reshape(-1, 2)
    tgt = np.asarray(tgt_xy, np.float64).reshape(-1, 2)
    f = _dens(f, src.shape[0])
    q = f * np.asarray(w, np.float64)[None, :]
    out = np.zeros((f.shape[0], tgt.shape[0]))
    step = max(1, _CHUNK_PAIRS // max(1, src.shape[0]))
    for i0 in range(0, tgt.shape[0], step):
        g = _kernel_block(src, tgt[i0:i0 + step], lam)
        for d in range(f.shape[0]):
            out[d, i0:i0 + step] = np.sum(g * q[d][None, :], axis=1)
    if csr is not None:
        A = _csr_matrix(csr, tgt.shape[0], src.shape[0])
        out += (A @ f.T).T
    return out


def adjoint(src_xy, w, g, tgt_xy, lam: float, csr=None) -> np.ndarray:
    """A^T g [ndens, n_src]."""
    src = np.asarray(src_xy, np.float64).reshape(-1, 2)
    tgt = np.asarray(tgt_xy, np.float64).reshape(-1, 2)
    g = _dens(g, tgt.shape[0])
    out = np.zeros((g.shape[0], src.shape[0]))
    step = max(1, _CHUNK_PAIRS // max(1, tgt.shape[0]))
    for j0 in range(0, src.shape[0], step):
        kb = _kernel_block(tgt, src[j0:j0 + step], lam)  # [src block, tgt]
        for d in range(g.shape[0]):
            out[d, j0:j0 + step] = np.sum(kb * g[d][None, :], axis=1)
    out *= np.asarray(w, np.float64)[None, :]
    if csr is not None:
        A = _csr_matrix(csr, tgt.shape[0], src.shape[0])
        out += (A.T @ g.T).T
    return out


def evaluate_rows(src_xy, w, f, tgt_xy, rows, lam: float, csr=None) -> np.ndarray:
    """V at the targets ``rows`` only ([ndens, len(rows)])."""
    rows = np.asarray(rows, np.int64)
    tgt = np.asarray(tgt_xy, np.float64).reshape(-1, 2)
    out = evaluate(src_xy, w, f, tgt[rows], lam)
    if csr is not None:
        rowptr, col, val = (np.asarray(a) for a in csr)
        fd = _dens(f, np.asarray(src_xy).reshape(-1, 2).shape[0])
        for k, i in enumerate(rows):
            a, b = int(rowptr[i]), int(rowptr[i + 1])
            out[:, k] += fd[:, col[a:b]] @ val[a:b]
    return out


def adjoint_cols(src_xy, w, g, tgt_xy, cols, lam: float, csr=None) -> np.ndarray:
    """A^T g at the sources ``cols`` only ([ndens, len(cols)])."""
    cols = np.asarray(cols, np.int64)
    src = np.asarray(src_xy, np.float64).reshape(-1, 2)
    out = adjoint(src[cols], np.asarray(w, np.float64)[cols], g, tgt_xy, lam)
    if csr is not None:
        gd = _dens(g, np.asarray(tgt_xy).reshape(-1, 2).shape[0])
        A = _csr_matrix(csr, gd.shape[1], src.shape[0])
        out += (A.T @ gd.T).T[:, cols]
    return out
