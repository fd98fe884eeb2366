"""Autotuner for the plan parameters of the volume-potential evaluation.

Picks the expansion order P (16, 24, 30), the leaf size (32, 64, 128) and the
density chunk (1, 2, 4, 8 densities per pass) that evaluate fastest while
keeping the relative l-infinity error (normalised by sum_j |w_j f_j|) below
`tol` times a safety factor. Accuracy is measured against the most accurate
configuration the library has (P = 30 with the all-FP64 kernels), on seeded
random densities, with the library itself; timing uses CUDA events around
graph-replayed evaluations. The correction matrix does not depend on these
parameters and is left out of the tuning runs.

Results are cached in a JSON file keyed by (geometry class, log2 of the point
count, number of densities).

tune_overlap picks, on a plan that carries its correction matrix, how much of
each SM the correction product takes while it runs beside the FMM.
"""

from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import vp

P_CHOICES = (16, 24, 30)
LEAF_CHOICES = (32, 64, 128)


def _cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "paper_2203_05933_gb300", "autotune.json")


def cache_key(geometry: str, n_points: int, ndens: int) -> str:
    return f"{geometry}|n2^{int(round(math.log2(max(n_points, 1))))}|d{ndens}"


def _load_cache(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(path, cache):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _time_eval(plan, f, out, steps):
    import torch

    stream = torch.cuda.current_stream()
    plan.eval(f, out=out)  # capture
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        plan.eval(f, out=out)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def tune(src_xy, w, tgt_xy, ndens: int = 1, geometry: str = "generic", root=None, tol: float = 1e-10,
         safety: float = 0.1, steps: int = 5, p_choices=P_CHOICES, leaf_choices=LEAF_CHOICES,
         use_cache: bool = True, seed: int = 7, flags: int = 0, f_check=None) -> dict:
    """Returns {"p_fmm", "leaf", "max_dens", "ms", "err", "table", "key", "cached"}.
    flags: the arithmetic of the plans tuned (0: float64, vp.VP_FLAG_FF: float-float).
    f_check: optional [k, n] densities of the workload itself, checked beside the
    random ones (the error is the larger of the two). Smooth densities have large
    multipole moments relative to sum |w f| and so show larger truncation errors
    than random ones; a choice made on random densities alone can miss the gate."""
    import torch

    n = int(np.asarray(src_xy).reshape(-1, 2).shape[0])
    key = cache_key(geometry, n, ndens) + f"|f{flags}"
    path = _cache_path()
    cache = _load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key], cached=True)
    rng = np.random.default_rng(seed)
    fr = rng.standard_normal((ndens, n))
    if f_check is not None:
        fc = np.asarray(f_check, np.float64).reshape(-1, n)[:max(1, min(ndens, 8))]
        k = min(fc.shape[0], ndens)
        fr[:k] = fc[:k] if ndens > 1 else fc[:1]
        if ndens == 1:
            fr = np.vstack([fr, rng.standard_normal((1, n))])  # one random density beside it
    nd_time = ndens  # timing uses the requested number of densities
    f = torch.as_tensor(fr, device="cuda")
    ndens = f.shape[0]
    wt = np.asarray(w, dtype=np.float64)
    norm = torch.as_tensor(np.abs(wt[None, :] * f.cpu().numpy()).sum(axis=1), device="cuda")
    chunk = 1
    while chunk * 2 <= min(ndens, 8):
        chunk *= 2
    ref_plan = vp.Plan.create(src_xy, w, tgt_xy, None, p_fmm=30, leaf=64, max_dens=chunk, flags=vp.VP_FLAG_FP64,
                              root=root)
    ref = ref_plan.eval(f)
    ref_plan.close()
    out = torch.empty_like(ref)
    ft, outt = f[:nd_time], out[:nd_time]
    table = []
    t0 = time.perf_counter()
    for P in p_choices:
        for leaf in leaf_choices:
            plan = vp.Plan.create(src_xy, w, tgt_xy, None, p_fmm=P, leaf=leaf, max_dens=chunk,
                                  flags=vp.VP_FLAG_GRAPH | flags, root=root)
            plan.eval(f, out=out)
            err = float(((out - ref).abs().max(dim=1).values / norm).max())
            ms = _time_eval(plan, ft, outt, steps)
            plan.close()
            table.append({"p_fmm": P, "leaf": leaf, "max_dens": chunk, "err": err, "ms": ms,
                          "ok": err <= tol * safety})
    ok = [r for r in table if r["ok"]]
    best = min(ok, key=lambda r: r["ms"]) if ok else max(table, key=lambda r: (r["p_fmm"], -r["ms"]))
    result = {"p_fmm": best["p_fmm"], "leaf": best["leaf"], "max_dens": best["max_dens"], "ms": best["ms"],
              "err": best["err"], "tol": tol, "safety": safety, "table": table, "key": key,
              "tuning_s": time.perf_counter() - t0}
    if use_cache:
        cache[key] = result
        _store_cache(path, cache)
    return dict(result, cached=False)


def tune_overlap(plan, f, out, choices=(0, 1, 2, 4), steps: int = 5) -> dict:
    """Time graph-replayed evaluations for each blocks-per-SM share of the
    correction product run beside the FMM (0: after it), keep the fastest.
    Returns {"blocks_per_sm", "table": [{"blocks_per_sm", "ms"}]}."""
    table = []
    for c in choices:
        plan.set_overlap(c)
        table.append({"blocks_per_sm": c, "ms": _time_eval(plan, f, out, steps)})
    best = min(table, key=lambda r: r["ms"])
    plan.set_overlap(best["blocks_per_sm"])
    return {"blocks_per_sm": best["blocks_per_sm"], "table": table}
