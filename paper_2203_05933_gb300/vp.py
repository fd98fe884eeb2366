"""Thin ctypes binding of libvp's C ABI (include/vp.h).

Each function carries the name of the C entry point it wraps and only marshals
arguments: torch tensors become device pointers, the current torch CUDA stream
becomes the stream argument, statuses become exceptions. Every step of the
computation runs in libvp's CUDA kernels. If libvp.so is missing the import of
this module's functions raises; there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

VP_OK = 0
VP_FLAG_TIMING = 1
VP_FLAG_FP64 = 2
VP_FLAG_GRAPH = 4
VP_FLAG_FF = 8
VP_KERNEL_LAPLACE = 0
VP_KERNEL_MHELMHOLTZ = 1

TREE_ARRAYS = {
    "box_level": 0, "box_ixy": 1, "box_parent": 2, "box_leaf": 3, "box_src": 4, "box_tgt": 5,
    "src_perm": 6, "tgt_perm": 7, "u_ptr": 8, "u_idx": 9, "v_ptr": 10, "v_idx": 11,
    "w_ptr": 12, "w_idx": 13, "x_ptr": 14, "x_idx": 15,
}

EXPORTED = [
    "vp_plan_create", "vp_plan_create_many", "vp_plan_create_upsampled", "vp_eval", "vp_eval_adjoint", "vp_eval_host", "vp_eval_batch",
    "vp_plan_info", "vp_plan_phase_times", "vp_plan_set_flags", "vp_plan_set_overlap", "vp_plan_destroy",
    "vp_green_eval_host",
    "vp_status_string", "vp_last_error", "vp_version", "vp_measure_peaks",
    "vp_tree_build", "vp_tree_build_device", "vp_tree_get", "vp_tree_destroy", "vp_interp_create", "vp_interp_eval", "vp_interp_destroy",
    "vp_tricorr_create", "vp_tricorr_eval", "vp_tricorr_near_eval", "vp_tricorr_destroy",
]


class VPError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = _load()
        msg = lib.vp_status_string(status).decode()
        detail = lib.vp_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){': ' + detail if detail else ''}")
        self.status = status


class vp_options(ctypes.Structure):
    _fields_ = [("p_fmm", ctypes.c_int32), ("leaf", ctypes.c_int32), ("max_level", ctypes.c_int32),
                ("max_dens", ctypes.c_int32), ("flags", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("root", ctypes.c_double * 3), ("lam", ctypes.c_double)]


class vp_plan_stats(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("n_tgt", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("p_fmm", ctypes.c_int32), ("leaf", ctypes.c_int32), ("max_dens", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("n_boxes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_u_pairs", ctypes.c_int64), ("n_v_pairs", ctypes.c_int64), ("n_w_pairs", ctypes.c_int64),
                ("n_x_pairs", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64), ("last_launches", ctypes.c_int64),
                ("n_problems", ctypes.c_int64), ("root", ctypes.c_double * 3), ("n_f", ctypes.c_int64),
                ("n_cells", ctypes.c_int64), ("sym_slots", ctypes.c_int64),
                ("p2p_evals", ctypes.c_int64), ("kernel", ctypes.c_int32), ("near_terms", ctypes.c_int32),
                ("lam", ctypes.c_double), ("near_ops", ctypes.c_int64)]


VP_UPS_DENSE = 0
VP_UPS_TENSOR = 1


class vp_upsample_type(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_q", ctypes.c_int32), ("n_p", ctypes.c_int32), ("qa", ctypes.c_int32),
                ("pa", ctypes.c_int32), ("qb", ctypes.c_int32), ("pb", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mat", ctypes.c_void_p), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p)]


class vp_interp_type(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_int32), ("order", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("coef", ctypes.c_void_p)]


class vp_upsample(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("types", ctypes.POINTER(vp_upsample_type)), ("n_cells", ctypes.c_int64),
                ("cell_type", ctypes.c_void_p), ("f_start", ctypes.c_void_p), ("src_start", ctypes.c_void_p)]


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libvp.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "vp_plan_create": [ctypes.POINTER(P), I64, P, P, I64, P, P, P, P, I64, ctypes.POINTER(vp_options), P],
        "vp_plan_create_many": [ctypes.POINTER(P), I32, P, P, P, P, P, P, P, P, P, P, ctypes.POINTER(vp_options), P],
        "vp_plan_create_upsampled": [ctypes.POINTER(P), I64, P, P, I64, P, P, P, P, I64, ctypes.POINTER(vp_upsample),
                                     ctypes.POINTER(vp_options), P],
        "vp_eval": [P, I32, P, I64, P, I64, P],
        "vp_eval_adjoint": [P, I32, P, I64, P, I64, P, I64, P, P],
        "vp_eval_host": [P, I32, P, P, P],
        "vp_eval_batch": [I32, P, P, P, P, P, P, P],
        "vp_plan_info": [P, ctypes.POINTER(vp_plan_stats)],
        "vp_plan_phase_times": [P, I32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(I32)],
        "vp_plan_destroy": [P],
        "vp_plan_set_flags": [P, ctypes.c_uint32],
        "vp_plan_set_overlap": [P, I32],
        "vp_green_eval_host": [I32, ctypes.c_double, I64, P, P],
        "vp_status_string": [I32],
        "vp_last_error": [],
        "vp_version": [],
        "vp_measure_peaks": [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), P],
        "vp_tree_build": [ctypes.POINTER(P), I64, P, I64, P, ctypes.POINTER(vp_options)],
        "vp_tree_build_device": [ctypes.POINTER(P), I64, P, I64, P, ctypes.POINTER(vp_options), P],
        "vp_tree_get": [P, I32, P, ctypes.POINTER(I64)],
        "vp_tree_destroy": [P],
        "vp_interp_create": [ctypes.POINTER(P), I32, ctypes.POINTER(vp_interp_type), I64, P, P, I64, P, P, P],
        "vp_interp_eval": [P, I32, P, I64, P, I64, P],
        "vp_interp_destroy": [P],
        "vp_tricorr_create": [ctypes.POINTER(P), I32, I32, I32, P, P, P, P, P, P, P],
        "vp_tricorr_eval": [P, I64, P, P, P],
        "vp_tricorr_near_eval": [P, I64, P, P, P, P],
        "vp_tricorr_destroy": [P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name in ("vp_status_string", "vp_last_error", "vp_version") else ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != VP_OK:
        raise VPError(status, where)


def make_options(p_fmm=0, leaf=0, max_level=0, max_dens=0, flags=0, root=None, kernel=0, lam=0.0) -> vp_options:
    o = vp_options()
    o.p_fmm, o.leaf, o.max_level, o.max_dens, o.flags = p_fmm, leaf, max_level, max_dens, flags
    o.kernel, o.lam = kernel, lam
    if root is not None:
        o.root[0], o.root[1], o.root[2] = root
    return o


def eval_batch(plans, fs, outs=None, stream=None):
    """vp_eval_batch: plans[k] evaluates fs[k] (CUDA float64 [ndens, n_src]) into
    outs[k] (allocated when None); returns the outputs."""
    import torch
    n = len(plans)
    if len(fs) != n:
        raise ValueError("one density block per plan")
    fs = [f.reshape(1, -1) if f.dim() == 1 else f for f in fs]
    fs = [f if f.stride(1) == 1 else f.contiguous() for f in fs]
    if outs is None:
        outs = [torch.empty((f.shape[0], p.n_tgt), dtype=torch.float64, device=f.device) for p, f in zip(plans, fs)]
    P = ctypes.c_void_p
    arr = lambda t, vals: (t * n)(*vals)
    _check(_load().vp_eval_batch(
        n, arr(P, [p.handle for p in plans]), arr(ctypes.c_int32, [f.shape[0] for f in fs]),
        arr(P, [f.data_ptr() for f in fs]), arr(ctypes.c_int64, [max(f.stride(0), f.shape[1], 1) for f in fs]),
        arr(P, [o.data_ptr() for o in outs]), arr(ctypes.c_int64, [max(o.stride(0), o.shape[1], 1) for o in outs]),
        _stream(stream)), "vp_eval_batch")
    return outs


def green_eval_host(r, kernel=0, lam=0.0):
    """G(r) of the kernel (VP_KERNEL_LAPLACE or VP_KERNEL_MHELMHOLTZ) at distances
    r > 0, on the host, with the plans' Bessel routines."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    g = np.empty_like(r)
    _check(_load().vp_green_eval_host(kernel, lam, r.size, r.ctypes.data_as(ctypes.c_void_p),
                                      g.ctypes.data_as(ctypes.c_void_p)), "vp_green_eval_host")
    return g


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f64(t, shape_last=None):
    import torch
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t, dtype=np.float64))
    t = t.to(device="cuda", dtype=torch.float64)
    return t.contiguous()


def vp_version() -> str:
    return _load().vp_version().decode()


def vp_status_string(status: int) -> str:
    return _load().vp_status_string(status).decode()


def vp_plan_create(src_xy, w, tgt_xy, csr=None, options: vp_options | None = None, stream=None):
    """Returns (plan handle, keep-alive tuple). Inputs may be numpy or torch."""
    import torch
    lib = _load()
    src = _dev_f64(src_xy).reshape(-1, 2)
    tgt = _dev_f64(tgt_xy).reshape(-1, 2)
    wt = _dev_f64(w).reshape(-1)
    if wt.numel() != src.shape[0]:
        raise ValueError("weights and sources differ in length")
    rowptr = col = val = None
    nnz = 0
    if csr is not None:
        r, c, v = csr
        rowptr = torch.as_tensor(np.asarray(r, dtype=np.int64) if not isinstance(r, torch.Tensor) else r)
        rowptr = rowptr.to(device="cuda", dtype=torch.int64).contiguous()
        col = torch.as_tensor(np.asarray(c, dtype=np.int32) if not isinstance(c, torch.Tensor) else c)
        col = col.to(device="cuda", dtype=torch.int32).contiguous()
        val = _dev_f64(v).reshape(-1)
        nnz = int(col.numel())
    h = ctypes.c_void_p()
    st = lib.vp_plan_create(ctypes.byref(h), src.shape[0], _ptr(src), _ptr(wt), tgt.shape[0], _ptr(tgt),
                            _ptr(rowptr), _ptr(col), _ptr(val), nnz,
                            ctypes.byref(options) if options is not None else None, _stream(stream))
    _check(st, "vp_plan_create")
    return h


def _csr_dev(csr):
    import torch
    if csr is None:
        return None, None, None, 0
    r, c, v = csr
    rowptr = torch.as_tensor(np.asarray(r, dtype=np.int64) if not isinstance(r, torch.Tensor) else r)
    rowptr = rowptr.to(device="cuda", dtype=torch.int64).contiguous()
    col = torch.as_tensor(np.asarray(c, dtype=np.int32) if not isinstance(c, torch.Tensor) else c)
    col = col.to(device="cuda", dtype=torch.int32).contiguous()
    val = _dev_f64(v).reshape(-1)
    return rowptr, col, val, int(col.numel())


def vp_plan_create_upsampled(src_xy, w, tgt_xy, csr, ups, options: vp_options | None = None, stream=None):
    """Plan of the oversampled smooth rule. src_xy, w: the q-nodes and their
    weights; csr columns index the p-nodes; ups: an object with `types` (dicts
    {"kind": "tensor", "a", "b"} or {"kind": "dense", "mat"}), `cell_type`,
    `f_start`, `src_start` (see setup.upsample.Upsampling)."""
    lib = _load()
    src = _dev_f64(src_xy).reshape(-1, 2)
    tgt = _dev_f64(tgt_xy).reshape(-1, 2)
    wt = _dev_f64(w).reshape(-1)
    if wt.numel() != src.shape[0]:
        raise ValueError("weights and sources differ in length")
    rowptr, col, val, nnz = _csr_dev(csr)
    keep = []
    nt = len(ups.types)
    tys = (vp_upsample_type * nt)()
    for k, ty in enumerate(ups.types):
        if ty["kind"] == "tensor":
            a = np.ascontiguousarray(ty["a"], np.float64)
            b = np.ascontiguousarray(ty["b"], np.float64)
            keep += [a, b]
            tys[k].kind = VP_UPS_TENSOR
            tys[k].qa, tys[k].pa = a.shape
            tys[k].qb, tys[k].pb = b.shape
            tys[k].n_q, tys[k].n_p = a.shape[0] * b.shape[0], a.shape[1] * b.shape[1]
            tys[k].a, tys[k].b = a.ctypes.data, b.ctypes.data
        else:
            m = np.ascontiguousarray(ty["mat"], np.float64)
            keep.append(m)
            tys[k].kind = VP_UPS_DENSE
            tys[k].n_q, tys[k].n_p = m.shape
            tys[k].mat = m.ctypes.data
    ct = np.ascontiguousarray(ups.cell_type, np.int32)
    fs = np.ascontiguousarray(ups.f_start, np.int64)
    ss = np.ascontiguousarray(ups.src_start, np.int64)
    u = vp_upsample()
    u.n_types = nt
    u.types = tys
    u.n_cells = ct.size
    u.cell_type, u.f_start, u.src_start = ct.ctypes.data, fs.ctypes.data, ss.ctypes.data
    h = ctypes.c_void_p()
    st = lib.vp_plan_create_upsampled(ctypes.byref(h), src.shape[0], _ptr(src), _ptr(wt), tgt.shape[0], _ptr(tgt),
                                      _ptr(rowptr), _ptr(col), _ptr(val), nnz, ctypes.byref(u),
                                      ctypes.byref(options) if options is not None else None, _stream(stream))
    _check(st, "vp_plan_create_upsampled")
    return h


def vp_plan_create_many(problems, options: vp_options | None = None, stream=None):
    """One plan for many independent problems. `problems` is a sequence of
    (src_xy, w, tgt_xy, csr or None, root or None); inputs may be numpy or torch."""
    import torch
    lib = _load()
    n = len(problems)
    keep = []
    ns = (ctypes.c_int64 * n)()
    nt = (ctypes.c_int64 * n)()
    nz = (ctypes.c_int64 * n)()
    ps, pw, pt = (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)()
    pr, pc, pv = (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)()
    roots = (ctypes.c_double * (3 * n))()
    any_csr = False
    for k, (src_xy, w, tgt_xy, csr, root) in enumerate(problems):
        src = _dev_f64(src_xy).reshape(-1, 2)
        tgt = _dev_f64(tgt_xy).reshape(-1, 2)
        wt = _dev_f64(w).reshape(-1)
        keep += [src, tgt, wt]
        ns[k], nt[k] = src.shape[0], tgt.shape[0]
        ps[k], pw[k], pt[k] = src.data_ptr(), wt.data_ptr(), tgt.data_ptr()
        if csr is not None:
            any_csr = True
            r = torch.as_tensor(np.asarray(csr[0], dtype=np.int64)).to("cuda").contiguous()
            c = torch.as_tensor(np.asarray(csr[1], dtype=np.int32)).to("cuda").contiguous()
            v = _dev_f64(csr[2]).reshape(-1)
            keep += [r, c, v]
            pr[k], pc[k], pv[k] = r.data_ptr(), c.data_ptr(), v.data_ptr()
            nz[k] = c.numel()
        if root is not None:
            roots[3 * k], roots[3 * k + 1], roots[3 * k + 2] = root
    h = ctypes.c_void_p()
    st = lib.vp_plan_create_many(ctypes.byref(h), n, ns, ps, pw, nt, pt,
                                 pr if any_csr else None, pc if any_csr else None, pv if any_csr else None,
                                 nz if any_csr else None, roots,
                                 ctypes.byref(options) if options is not None else None, _stream(stream))
    _check(st, "vp_plan_create_many")
    return h


def vp_eval(plan, f, out=None, stream=None):
    """f: CUDA float64 tensor [ndens, n_src] (or [n_src]); returns out [ndens, n_tgt]."""
    import torch
    lib = _load()
    squeeze = f.dim() == 1
    f2 = f.reshape(1, -1) if squeeze else f
    if f2.stride(1) != 1:
        f2 = f2.contiguous()
    info = vp_plan_info(plan)
    if out is None:
        out = torch.empty((f2.shape[0], info.n_tgt), dtype=torch.float64, device=f2.device)
    ld_f = max(f2.stride(0), f2.shape[1], 1)
    ld_out = max(out.stride(0), out.shape[1], 1)
    st = lib.vp_eval(plan, f2.shape[0], _ptr(f2), ld_f, _ptr(out), ld_out, _stream(stream))
    _check(st, "vp_eval")
    return out[0] if squeeze else out


def vp_eval_adjoint(plan, g, grad_f=True, f=None, grad_tgt=False, stream=None):
    """Returns (grad_f [ndens, n_src] or None, grad_tgt [n_tgt, 2] or None)."""
    import torch
    lib = _load()
    g2 = g.reshape(1, -1) if g.dim() == 1 else g
    g2 = g2.contiguous()
    info = vp_plan_info(plan)
    nd = g2.shape[0]
    gf = torch.empty((nd, info.n_f), dtype=torch.float64, device=g2.device) if grad_f else None
    gt = torch.empty((info.n_tgt, 2), dtype=torch.float64, device=g2.device) if grad_tgt else None
    f2 = None
    if grad_tgt:
        if f is None:
            raise ValueError("the target gradient needs f")
        f2 = (f.reshape(1, -1) if f.dim() == 1 else f).contiguous()
    st = lib.vp_eval_adjoint(plan, nd, _ptr(g2), max(info.n_tgt, 1), _ptr(gf), max(info.n_f, 1),
                             _ptr(f2), max(info.n_f, 1), _ptr(gt), _stream(stream))
    _check(st, "vp_eval_adjoint")
    if gf is not None and g.dim() == 1:
        gf = gf[0]
    return gf, gt


def vp_eval_host(plan, f_host: np.ndarray, out_host: np.ndarray | None = None, stream=None) -> np.ndarray:
    """Host-buffer evaluation: f_host [ndens, n_src] float64 (pinned or pageable)."""
    lib = _load()
    info = vp_plan_info(plan)
    f_host = np.ascontiguousarray(f_host, dtype=np.float64).reshape(-1, info.n_f) if info.n_f else \
        np.zeros((np.asarray(f_host).reshape(-1, 0).shape[0], 0))
    nd = f_host.shape[0]
    if out_host is None:
        out_host = np.empty((nd, info.n_tgt), np.float64)
    st = lib.vp_eval_host(plan, nd, f_host.ctypes.data_as(ctypes.c_void_p),
                          out_host.ctypes.data_as(ctypes.c_void_p), _stream(stream))
    _check(st, "vp_eval_host")
    return out_host


def vp_eval_host_ptr(plan, ndens: int, f_ptr: int, out_ptr: int, stream=None):
    """vp_eval_host on raw host addresses (e.g. pinned torch tensors)."""
    st = _load().vp_eval_host(plan, ndens, ctypes.c_void_p(f_ptr), ctypes.c_void_p(out_ptr), _stream(stream))
    _check(st, "vp_eval_host")


def vp_plan_info(plan) -> vp_plan_stats:
    s = vp_plan_stats()
    _check(_load().vp_plan_info(plan, ctypes.byref(s)), "vp_plan_info")
    return s


def vp_plan_phase_times(plan) -> dict:
    lib = _load()
    cap = 32
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    n = ctypes.c_int32()
    _check(lib.vp_plan_phase_times(plan, cap, names, ms, ctypes.byref(n)), "vp_plan_phase_times")
    return {names[i].decode(): ms[i] for i in range(min(n.value, cap))}


def vp_plan_set_flags(plan, flags: int):
    _check(_load().vp_plan_set_flags(plan, flags), "vp_plan_set_flags")


def vp_plan_destroy(plan):
    if plan:
        _check(_load().vp_plan_destroy(plan), "vp_plan_destroy")


def vp_tree_build(src_xy: np.ndarray, tgt_xy: np.ndarray, options: vp_options | None = None) -> dict:
    """Host tree + interaction lists for inspection; returns a dict of int32 arrays."""
    lib = _load()
    src = np.ascontiguousarray(src_xy, np.float64).reshape(-1, 2)
    tgt = np.ascontiguousarray(tgt_xy, np.float64).reshape(-1, 2)
    h = ctypes.c_void_p()
    st = lib.vp_tree_build(ctypes.byref(h), src.shape[0], src.ctypes.data_as(ctypes.c_void_p), tgt.shape[0],
                           tgt.ctypes.data_as(ctypes.c_void_p),
                           ctypes.byref(options) if options is not None else None)
    _check(st, "vp_tree_build")
    return _tree_arrays(h)


def vp_tree_build_device(src_xy, tgt_xy, options: vp_options | None = None, stream=None) -> dict:
    """The same tree and lists built on the GPU (vp_tree_build_device) from device
    copies of the points; returns the same dict of int32 arrays."""
    lib = _load()
    src = _dev_f64(src_xy).reshape(-1, 2)
    tgt = _dev_f64(tgt_xy).reshape(-1, 2)
    h = ctypes.c_void_p()
    st = lib.vp_tree_build_device(ctypes.byref(h), src.shape[0], _ptr(src), tgt.shape[0], _ptr(tgt),
                                  ctypes.byref(options) if options is not None else None, _stream(stream))
    _check(st, "vp_tree_build_device")
    return _tree_arrays(h)


def _tree_arrays(h) -> dict:
    lib = _load()
    out = {}
    try:
        for name, which in TREE_ARRAYS.items():
            n = ctypes.c_int64()
            _check(lib.vp_tree_get(h, which, None, ctypes.byref(n)), "vp_tree_get")
            a = np.empty(n.value, np.int32)
            _check(lib.vp_tree_get(h, which, a.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)), "vp_tree_get")
            if name in ("box_ixy", "box_src", "box_tgt"):
                a = a.reshape(-1, 2)
            out[name] = a
    finally:
        lib.vp_tree_destroy(h)
    return out


@dataclass
class Plan:
    """Owning wrapper: creates the plan, destroys it when closed or collected."""

    handle: ctypes.c_void_p
    n_src: int
    n_tgt: int
    n_f: int = -1  # density length (n_src unless upsampled)

    def __post_init__(self):
        if self.n_f < 0:
            self.n_f = self.n_src

    @classmethod
    def create(cls, src_xy, w, tgt_xy, csr=None, p_fmm=0, leaf=0, max_level=0, max_dens=0, flags=0,
               root=None, stream=None, kernel=0, lam=0.0) -> "Plan":
        """kernel: VP_KERNEL_LAPLACE (default) or VP_KERNEL_MHELMHOLTZ with parameter lam."""
        opts = make_options(p_fmm, leaf, max_level, max_dens, flags, root, kernel, lam)
        h = vp_plan_create(src_xy, w, tgt_xy, csr, opts, stream)
        info = vp_plan_info(h)
        return cls(h, int(info.n_src), int(info.n_tgt))

    @classmethod
    def create_many(cls, problems, p_fmm=0, leaf=0, max_level=0, max_dens=0, flags=0, stream=None) -> "Plan":
        """problems: sequence of (src_xy, w, tgt_xy, csr or None, root or None)."""
        opts = make_options(p_fmm, leaf, max_level, max_dens, flags, None)
        h = vp_plan_create_many(problems, opts, stream)
        info = vp_plan_info(h)
        return cls(h, int(info.n_src), int(info.n_tgt))

    @classmethod
    def create_upsampled(cls, src_xy, w, tgt_xy, csr, ups, p_fmm=0, leaf=0, max_level=0, max_dens=0, flags=0,
                         root=None, stream=None) -> "Plan":
        """Oversampled smooth rule: src_xy, w are the q-nodes; densities live on the
        p-nodes described by ups (setup.upsample.Upsampling)."""
        opts = make_options(p_fmm, leaf, max_level, max_dens, flags, root)
        h = vp_plan_create_upsampled(src_xy, w, tgt_xy, csr, ups, opts, stream)
        info = vp_plan_info(h)
        return cls(h, int(info.n_src), int(info.n_tgt), int(info.n_f))

    def eval(self, f, out=None, stream=None):
        return vp_eval(self.handle, f, out, stream)

    def adjoint(self, g, grad_f=True, f=None, grad_tgt=False, stream=None):
        return vp_eval_adjoint(self.handle, g, grad_f, f, grad_tgt, stream)

    def eval_host(self, f_host, out_host=None, stream=None):
        return vp_eval_host(self.handle, f_host, out_host, stream)

    def set_flags(self, flags: int):
        vp_plan_set_flags(self.handle, flags)

    def set_overlap(self, blocks_per_sm: int):
        _check(_load().vp_plan_set_overlap(self.handle, blocks_per_sm), "vp_plan_set_overlap")

    def info(self) -> vp_plan_stats:
        return vp_plan_info(self.handle)

    def phase_times(self) -> dict:
        return vp_plan_phase_times(self.handle)

    def close(self):
        if self.handle:
            vp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vp_measure_peaks(stream=None, tensor=False):
    """Binding of vp_measure_peaks: (FP64, FP32) FMA throughput of the current
    device in TFLOP/s; with tensor=True also (f64 mma, bf16 mma) throughput in
    TFLOP/s and int8 mma throughput in T ops/s, returned as a 5-tuple."""
    lib = _load()
    a, b, c, d, e = (ctypes.c_double() for _ in range(5))
    _check(lib.vp_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c) if tensor else None,
                                ctypes.byref(d) if tensor else None, ctypes.byref(e) if tensor else None,
                                _stream(stream)), "vp_measure_peaks")
    return (a.value, b.value, c.value, d.value, e.value) if tensor else (a.value, b.value)


def vp_eval_direct_static(src_xy, w, f, tgt_xy, out, csr=None, stream=None):
    """Binding of the allocation-free entry point (direct sum, scratch in a fixed
    device array). Every argument must already be a CUDA float64 tensor (CSR:
    int64 rowptr, int32 col, float64 val) because the call itself allocates
    nothing; `out` [ndens, n_tgt] receives the result."""
    import torch

    lib = _load()
    fn = lib.vp_eval_direct_static
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    fn.argtypes = [I64, P, P, I32, P, I64, I64, P, P, P, P, P, I64, P]
    fn.restype = ctypes.c_int
    rowptr, col, val = csr if csr is not None else (None, None, None)

    def need(t, name, dtype, shape_ok):
        # the call allocates nothing, so nothing is copied or converted here
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if t.numel() > 0 and t.stride(-1) != 1:
            raise ValueError(f"{name} must have unit stride in its last dimension")
        if not shape_ok(t):
            raise ValueError(f"{name} has shape {tuple(t.shape)}")

    need(src_xy, "src_xy", torch.float64, lambda t: t.dim() == 2 and t.shape[1] == 2 and t.is_contiguous())
    need(tgt_xy, "tgt_xy", torch.float64, lambda t: t.dim() == 2 and t.shape[1] == 2 and t.is_contiguous())
    n_src, n_tgt = src_xy.shape[0], tgt_xy.shape[0]
    need(w, "w", torch.float64, lambda t: t.dim() == 1 and t.shape[0] == n_src)
    f2 = f.reshape(1, -1) if f.dim() == 1 else f
    out2 = out.reshape(1, -1) if out.dim() == 1 else out
    need(f2, "f", torch.float64, lambda t: t.dim() == 2 and t.shape[1] == n_src)
    need(out2, "out", torch.float64, lambda t: t.dim() == 2 and t.shape[1] == n_tgt and t.shape[0] == f2.shape[0])
    if csr is not None:
        need(rowptr, "csr rowptr", torch.int64, lambda t: t.dim() == 1 and t.shape[0] == n_tgt + 1)
        need(col, "csr col", torch.int32, lambda t: t.dim() == 1)
        need(val, "csr val", torch.float64, lambda t: t.dim() == 1 and t.shape[0] == col.shape[0])
    ld_f = f2.stride(0) if f2.shape[0] > 1 else max(n_src, 1)
    ld_out = out2.stride(0) if out2.shape[0] > 1 else max(n_tgt, 1)
    st = fn(n_src, _ptr(src_xy), _ptr(w), f2.shape[0], _ptr(f2), ld_f, n_tgt, _ptr(tgt_xy),
            _ptr(rowptr), _ptr(col), _ptr(val), _ptr(out2), ld_out, _stream(stream))
    _check(st, "vp_eval_direct_static")
    return out


class Interp:
    """Interpolation of nodal values to points inside cells (vp_interp_*).
    types: [(basis, order, C)] with basis 0 (tensor Legendre, boxes) or 1
    (simplex); cell_type [n_cells]; node_start [n_cells + 1]; pt_cell [n_pts];
    pt_ref [n_pts, 2] reference coordinates."""

    def __init__(self, types, cell_type, node_start, pt_cell, pt_ref, stream=None):
        import torch
        lib = _load()
        keep = []
        tys = (vp_interp_type * len(types))()
        for k, (basis, order, C) in enumerate(types):
            c = np.ascontiguousarray(C, np.float64)
            keep.append(c)
            tys[k].basis, tys[k].order, tys[k].n_nodes = basis, order, c.shape[0]
            tys[k].coef = c.ctypes.data
        ct = np.ascontiguousarray(cell_type, np.int32)
        ns = np.ascontiguousarray(node_start, np.int64)
        pc = torch.as_tensor(np.ascontiguousarray(pt_cell, np.int32)).to("cuda")
        pr = _dev_f64(pt_ref).reshape(-1, 2)
        h = ctypes.c_void_p()
        st = lib.vp_interp_create(ctypes.byref(h), len(types), tys, ct.size, ct.ctypes.data_as(ctypes.c_void_p),
                                  ns.ctypes.data_as(ctypes.c_void_p), pc.numel(), _ptr(pc), _ptr(pr), _stream(stream))
        _check(st, "vp_interp_create")
        self.handle = h
        self.n_pts = int(pc.numel())
        self.n_vals = int(ns[-1])

    def eval(self, v, out=None, stream=None):
        """v: CUDA float64 [ndens, n_vals] (or [n_vals]); returns [ndens, n_pts]."""
        import torch
        squeeze = v.dim() == 1
        v2 = (v.reshape(1, -1) if squeeze else v).contiguous()
        if out is None:
            out = torch.empty((v2.shape[0], self.n_pts), dtype=torch.float64, device=v2.device)
        st = _load().vp_interp_eval(self.handle, v2.shape[0], _ptr(v2), max(v2.shape[1], 1), _ptr(out),
                                    max(out.stride(0), self.n_pts, 1), _stream(stream))
        _check(st, "vp_interp_eval")
        return out[0] if squeeze else out

    def close(self):
        if self.handle:
            _check(_load().vp_interp_destroy(self.handle), "vp_interp_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TriCorr:
    """Self- and near-singular correction blocks of mapped triangles on the GPU (vp_tricorr_*).
    rules: dict of setup.tricorr.self_rules (xi, eta, tw, C, chi, tau, B)."""

    def __init__(self, rules, stream=None):
        lib = _load()
        ref = np.ascontiguousarray(np.stack([rules["xi"], rules["eta"]], axis=1), np.float64)
        arrs = [ref, np.ascontiguousarray(rules["tw"], np.float64), np.ascontiguousarray(rules["C"], np.float64),
                np.ascontiguousarray(rules["chi"], np.float64), np.ascontiguousarray(rules["tau"], np.float64),
                np.ascontiguousarray(rules["B"], np.float64)]
        n_nodes, n_basis, n_rule = ref.shape[0], arrs[2].shape[0], arrs[3].shape[1]
        h = ctypes.c_void_p()
        st = lib.vp_tricorr_create(ctypes.byref(h), n_nodes, n_basis, n_rule,
                                   *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs], _stream(stream))
        _check(st, "vp_tricorr_create")
        self.handle = h
        self.n_nodes = n_nodes

    def eval(self, geom, out=None, stream=None):
        """geom: [n_cells, 12] (numpy or CUDA tensor); returns [n_cells, n_nodes, n_nodes]."""
        import torch
        g = _dev_f64(geom).reshape(-1, 12)
        if out is None:
            out = torch.empty((g.shape[0], self.n_nodes, self.n_nodes), dtype=torch.float64, device=g.device)
        _check(_load().vp_tricorr_eval(self.handle, g.shape[0], _ptr(g), _ptr(out), _stream(stream)), "vp_tricorr_eval")
        return out

    def near(self, geom, tgt, out=None, stream=None):
        """Near-singular block rows (vp_tricorr_near_eval): geom [n_pairs, 12] the cell
        of each pair, tgt [n_pairs, 2] its target outside the cell (numpy or CUDA
        tensors); returns [n_pairs, n_nodes]."""
        import torch
        g = _dev_f64(geom).reshape(-1, 12)
        t = _dev_f64(tgt).reshape(-1, 2)
        if t.shape[0] != g.shape[0]:
            raise ValueError("one target per cell")
        if out is None:
            out = torch.empty((g.shape[0], self.n_nodes), dtype=torch.float64, device=g.device)
        _check(_load().vp_tricorr_near_eval(self.handle, g.shape[0], _ptr(g), _ptr(t), _ptr(out), _stream(stream)),
               "vp_tricorr_near_eval")
        return out

    def close(self):
        if self.handle:
            _check(_load().vp_tricorr_destroy(self.handle), "vp_tricorr_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
