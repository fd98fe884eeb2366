"""Benchmark of the volume-potential hot path on GB300.

One step = one vp_eval of the unit-disk workload (about 1.1 M quadrature nodes of
adaptive boxes and curved triangles, targets = nodes, self + near-cell
correction matrix of about 6e8 nonzeros): charges, the whole FMM (P2M, M2M,
M2L, L2L, L2P, M2P, P2L, P2P) and the correction apply.

Metric: volume-potential Mpoints/s = n_targets * ndens / t_eval, FP64, with the
relative l-infinity error against the CPU oracle (sampled targets) reported
beside it (the gate is 1e-10, normalised by sum_j |w_j f_j|).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch under torch.distributed.run; every rank evaluates its own
independent disk problem (different seeded refinement), no data-path
collective (weak scaling).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "volume-potential Mpoints/s (FP64, rel err <=1e-10), batched/adjoint vs plain FMM"
UNIT = "Mpoints/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # 2 FP64 FMA/clk/SM (measured), 152 SMs, 2070 MHz
FP32_OPS_PEAK = 152 * 128 * 2.070e9 / 1e12     # FP32/INT32 lane-operations per second (T ops/s)
P2P_FLOP_PER_PAIR = 27.0  # 7 flops + 20 flop-equivalents for one FP64 log (stated convention)
P2P_FF_OPS_PER_PAIR = 77.0  # FP32 operations of the float-float pair evaluation (k_leaf_ff, exact-hi pairs)
P2P_FF_OPS_REVERSE = 14.0   # extra FP32 operations when one evaluation serves both directions (symmetric near field)
# DRAM bytes (read + write) per work unit from one ncu capture of the current
# kernels on the medium disk case (profiles/*_disk_medium.md), scaled to a
# launch by the units it processes; None once a kernel changes until re-profiled.
PROFILED_TRAFFIC = {
    "leaf": ((15.194368e6 + 1024) / 84050308, "evaluated distances", "profiles/k_leaf_ff_sym_disk_medium.md"),
    "m2l": (3.043e6 / 145118, "V-list pairs", "profiles/k_m2l_ff_disk_medium.md"),
    "out": ((1298.617e6 + 5.689e6) / 159866880, "nonzeros", "profiles/k_out_grouped_disk_medium.md"),
}


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "profiling-recipe fallback 6.8 TB/s"


def roofline_models(info, prob, ndens=1):
    """Per-phase roofline models: algorithmic work per launch of each phase."""
    P = info.p_fmm
    hbm, hbm_src = hbm_peak()
    evals = int(info.p2p_evals)
    two_way = int(info.p2p_pairs) - evals  # evaluations that serve both directions
    return {
        "leaf": {"bound": "alu", "kernel": "k_leaf_ff (float-float P2P + FP64 L2P/M2P)",
                 "work": (evals * P2P_FF_OPS_PER_PAIR + two_way * P2P_FF_OPS_REVERSE) * ndens, "unit": "T FP32-ops/s",
                 "peak": FP32_OPS_PEAK, "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz",
                 "fp64_equiv_flop": (evals * P2P_FLOP_PER_PAIR + two_way * 7.0) * ndens, "units": evals,
                 "per_unit": f"{P2P_FF_OPS_PER_PAIR:.0f} FP32 ops per evaluated source-target distance, "
                             f"+{P2P_FF_OPS_REVERSE:.0f} when it serves both directions "
                             f"({evals} evaluations for {info.p2p_pairs} directed pairs)"},
        "m2l": {"bound": "alu", "kernel": "k_m2l_ff (float-float scaled-Hankel M2L)",
                "work": info.n_v_pairs * (P + 1) * (24.0 * P + 100.0) * ndens, "unit": "T FP32-ops/s",
                "peak": FP32_OPS_PEAK, "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz",
                "fp64_equiv_flop": info.n_v_pairs * 8.0 * (P + 1) ** 2 * ndens, "units": info.n_v_pairs,
                "per_unit": f"(P+1)(24P+100) FP32 ops per V-list pair, P={P}"},
        "out": {"bound": "hbm", "kernel": "k_out_grouped (correction apply, rows grouped by shared column lists)",
                "work": info.nnz * 8.0 + info.n_tgt * 8.0 * (2 * ndens + 1), "unit": "GB/s",
                "peak": hbm, "peak_source": hbm_src, "units": info.nnz,
                "per_unit": "8 B per nonzero (one 64-bit value) + 8 B per row per density in and out"},
    }


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--p", type=int, default=0, help="expansion order (0: autotuned with the leaf size)")
    ap.add_argument("--leaf", type=int, default=0, help="leaf size (0: autotuned with the expansion order)")
    ap.add_argument("--batched", type=int, default=64, help="densities of the batched leg (0: skip)")
    ap.add_argument("--size", default="full", choices=["full", "medium", "small"],
                    help="disk levels 7-9 (1.1 M nodes), 6-8 (profiling) or 5-7")
    ap.add_argument("--many", type=int, default=256, help="problems of the many-problem leg (0: skip)")
    ap.add_argument("--star", type=int, default=1, help="run the 4 M star-with-holes leg (0: skip)")
    ap.add_argument("--upsampled", type=int, default=1, help="run the oversampled (q = 2p) disk leg (0: skip)")
    ap.add_argument("--tricorr", type=int, default=1, help="run the triangle self-correction leg (0: skip)")
    ap.add_argument("--mhelm", type=float, default=100.0,
                    help="lambda^2 of the modified-Helmholtz disk leg (0: skip)")
    ap.add_argument("--interp", type=int, default=1 << 20,
                    help="random points of the interpolation leg (0: skip)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Seed of the disk problem of one replica (each rank refines around its own bumps)."""
    from paper_2203_05933_gb300 import inputs

    return inputs.SEED_BASE + 2 + 1000 * rank


def combine_ranks(t_dev: float, points: float, world: int, device) -> tuple[float, float]:
    """Whole-job figures of a replica run: the slowest rank's device time (max) and
    the points all ranks evaluated (sum). One process per GPU; any
    torch.distributed backend (NCCL on the GPUs, gloo in the CPU tests)."""
    if world <= 1:
        return t_dev, points
    import torch
    import torch.distributed as dist

    t = torch.tensor([t_dev], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([points], dtype=torch.float64, device=device)
    dist.all_reduce(p)
    return float(t.item()), float(p.item())


def make_problem(args, rank):
    from paper_2203_05933_gb300 import inputs

    seed = rank_seed(rank)
    if args.size == "small":
        return inputs.disk_problem(base_level=5, fine_level=7, seed=seed, name="disk_small")
    if args.size == "medium":
        return inputs.disk_problem(base_level=6, fine_level=8, seed=seed, name="disk_medium")
    return inputs.disk_problem(seed=seed, name="disk_1M")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def flush_l2(buf):
    buf.add_(1.0)  # writes 256 MB, twice the 129 MB L2


def run_reference(args, rank, world):
    """The oracle (plain C, OpenMP) on the host cores: each step evaluates a
    bounded seeded sample of targets of the same workload, exactly."""
    if rank != 0:
        return
    import oracle
    from paper_2203_05933_gb300 import inputs

    oracle.build()
    prob = make_problem(args, 0)
    rng = np.random.default_rng(7)
    cores = oracle.max_threads()
    sample = 256
    rows = rng.choice(prob.n_tgt, size=sample, replace=False)
    csr = oracle.csr_rows(prob.csr, rows)
    tgt = prob.tgt_xy[rows]
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.evaluate(prob.src_xy, prob.w, prob.f, tgt, csr)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = sample * prob.ndens / t / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": prob.name, "n_src": prob.n_src, "n_tgt": prob.n_tgt, "nnz": prob.nnz,
                   "ndens": prob.ndens, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} seeded targets of {prob.n_tgt} per step, full direct sum over "
                                   f"{prob.n_src} sources + their correction rows"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(prob, out_gpu=None, budget_s=15.0):
    """The oracle timed on a bounded seeded sample of targets (about budget_s of
    host work, all host cores). Its values at those targets also give the GPU
    result's relative error there (out_gpu: [ndens, n_tgt] host copy), so the
    oracle runs in this leg only. Returns (record, rel_err or None)."""
    import oracle
    from paper_2203_05933_gb300 import inputs

    oracle.build()
    cores = oracle.max_threads()
    rng = np.random.default_rng(11)
    probe = 32
    rows = rng.choice(prob.n_tgt, size=probe, replace=False)
    t0 = time.perf_counter()
    oracle.evaluate(prob.src_xy, prob.w, prob.f[:1], prob.tgt_xy[rows], oracle.csr_rows(prob.csr, rows))
    per_tgt = (time.perf_counter() - t0) / probe
    n = int(min(max(budget_s / max(per_tgt, 1e-9), 64), 16384))
    rows = rng.choice(prob.n_tgt, size=n, replace=False)
    t0 = time.perf_counter()
    ref = oracle.evaluate(prob.src_xy, prob.w, prob.f[:1], prob.tgt_xy[rows], oracle.csr_rows(prob.csr, rows))
    dt = time.perf_counter() - t0
    err = None
    if out_gpu is not None:
        err = float(np.max(np.abs(out_gpu[:1, rows] - ref) / inputs.normaliser(prob)[:1, None]))
    return ({"value": n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"{n} seeded targets of {prob.n_tgt}, full direct sum over {prob.n_src} sources + "
                       f"correction rows, one density ({dt:.1f} s)"}, err)


def cpu_baseline_mhelm(prob, lam, out_gpu, budget_s=8.0):
    """The modified-Helmholtz oracle on a bounded seeded sample of targets (about
    budget_s of host work); also gives the GPU result's relative error there,
    normalised by (lambda^2/2pi) sum_j |w_j f_j|. Returns (record, rel_err)."""
    from oracle import mhelm
    from paper_2203_05933_gb300 import inputs

    rng = np.random.default_rng(12)
    probe = 8
    rows = rng.choice(prob.n_tgt, size=probe, replace=False)
    t0 = time.perf_counter()
    mhelm.evaluate_rows(prob.src_xy, prob.w, prob.f[:1], prob.tgt_xy, rows, lam, prob.csr)
    per_tgt = (time.perf_counter() - t0) / probe
    n = int(min(max(budget_s / max(per_tgt, 1e-9), 32), 4096))
    rows = rng.choice(prob.n_tgt, size=n, replace=False)
    t0 = time.perf_counter()
    ref = mhelm.evaluate_rows(prob.src_xy, prob.w, prob.f[:1], prob.tgt_xy, rows, lam, prob.csr)
    dt = time.perf_counter() - t0
    scale = lam * lam / (2 * math.pi) * inputs.normaliser(prob)[:1, None]
    err = float(np.max(np.abs(out_gpu[:1, rows] - ref) / scale))
    return ({"value": n / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
             "sample": f"{n} seeded targets of {prob.n_tgt}, direct sum with scipy K0 over {prob.n_src} sources "
                       f"+ correction rows ({dt:.1f} s)"}, err)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2203_05933_gb300 import build, vp

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    vp._load()
    prob = make_problem(args, rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    tuned = None
    if args.p == 0 or args.leaf == 0:
        from paper_2203_05933_gb300 import autotune
        tuned = autotune.tune(prob.src_xy, prob.w, prob.tgt_xy, ndens=1, geometry=prob.name, root=prob.root,
                              use_cache=False, steps=3)
        args.p = args.p or tuned["p_fmm"]
        args.leaf = args.leaf or tuned["leaf"]
    plan = vp.Plan.create(prob.src_xy, prob.w, prob.tgt_xy, prob.csr, p_fmm=args.p, leaf=args.leaf,
                          max_dens=8, flags=vp.VP_FLAG_GRAPH, root=prob.root)
    info = plan.info()
    f = torch.as_tensor(prob.f, device=dev)
    out = torch.empty((prob.ndens, prob.n_tgt), dtype=torch.float64, device=dev)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)

    overlap = None
    if tuned is not None and prob.csr is not None:
        from paper_2203_05933_gb300 import autotune
        overlap = autotune.tune_overlap(plan, f, out, choices=(0, 1, 2, 4, 8))

    # first evaluation; its result is checked against the oracle in the CPU-baseline leg
    plan.eval(f, out=out)
    torch.cuda.synchronize()
    out_first = out.cpu().numpy() if rank == 0 else None

    def timed(fn, steps):
        """CUDA-event time of each call on the evaluation stream, L2 flushed before each."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush_l2(flush)
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) / 1e3 for a, b in ev]

    for _ in range(args.warmup):
        flush_l2(flush)
        plan.eval(f, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_s = timed(lambda: plan.eval(f, out=out), args.steps)
    wall = time.perf_counter() - wall0
    t_dev = sum(step_s)
    launches_per_eval = plan.info().last_launches
    t_dev, pts = combine_ranks(t_dev, float(prob.n_tgt * prob.ndens * args.steps), world, dev)
    value = pts / t_dev / 1e6

    # per-phase CUDA-event times (same kernels launched one by one, timing events on the stream)
    plan.set_flags(vp.VP_FLAG_TIMING)
    phase_sum = {}
    for k in range(args.steps):
        flush_l2(flush)
        plan.eval(f, out=out)
        for name, ms in plan.phase_times().items():
            phase_sum[name] = phase_sum.get(name, 0.0) + ms
    plan.set_flags(vp.VP_FLAG_GRAPH)
    phase_ms = {k: v / args.steps for k, v in phase_sum.items()}

    # e2e: the C-ABI host-buffer entry point, pinned buffers, copies inside the timed region
    f_pin = torch.empty((prob.ndens, prob.n_src), dtype=torch.float64, pin_memory=True)
    f_pin.copy_(torch.as_tensor(prob.f))
    o_pin = torch.empty((prob.ndens, prob.n_tgt), dtype=torch.float64, pin_memory=True)
    vp.vp_eval_host_ptr(plan.handle, prob.ndens, f_pin.data_ptr(), o_pin.data_ptr())
    e2e_t = []
    for k in range(max(3, args.steps // 2)):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vp.vp_eval_host_ptr(plan.handle, prob.ndens, f_pin.data_ptr(), o_pin.data_ptr())
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = prob.n_tgt * prob.ndens / float(np.mean(e2e_t)) / 1e6
    clk = clocks.stop()

    # batched leg: many densities through one plan (chunks of 8 densities per pass)
    batched = None
    if args.batched > 0:
        rng = np.random.default_rng(3)
        fb = torch.as_tensor(rng.standard_normal((args.batched, prob.n_src)), device=dev)
        ob = torch.empty((args.batched, prob.n_tgt), dtype=torch.float64, device=dev)
        bovl = None
        if overlap is not None:  # the share beside the FMM, tuned for passes of 8 densities
            from paper_2203_05933_gb300 import autotune
            bovl = autotune.tune_overlap(plan, fb, ob, choices=(0, 2, 4, 8), steps=2)
        plan.eval(fb, out=ob)
        bt = timed(lambda: plan.eval(fb, out=ob), max(2, args.steps // 5))
        if overlap is not None:
            plan.set_overlap(overlap["blocks_per_sm"])
        bv = prob.n_tgt * args.batched / float(np.mean(bt)) / 1e6
        # per-phase times of one pass of 8 densities
        plan.set_flags(vp.VP_FLAG_TIMING)
        flush_l2(flush)
        plan.eval(fb[:8], out=ob[:8])
        bphase = plan.phase_times()
        plan.set_flags(vp.VP_FLAG_GRAPH)
        batched = {"ndens": args.batched, "value": bv, "unit": UNIT, "speedup_vs_single": bv / value,
                   "ms_per_step": float(np.mean(bt)) * 1e3, "phase_ms_8_densities": bphase, "overlap": bovl}
        del fb, ob

    # adjoint leg: transposed FMM + transposed correction (dL/df), one density
    g = torch.as_tensor(np.random.default_rng(4).standard_normal((1, prob.n_tgt)), device=dev)
    plan.adjoint(g)
    at = timed(lambda: plan.adjoint(g), max(2, args.steps // 5))
    adjoint = {"value": prob.n_src / float(np.mean(at)) / 1e6, "unit": "Msources/s",
               "ms_per_step": float(np.mean(at)) * 1e3, "ratio_vs_forward": (t_dev / args.steps) / float(np.mean(at))}

    # many-problem leg: 256 uneven square and disk problems in one plan, one graph per evaluation
    many = None
    if args.many > 0 and rank == 0:
        from paper_2203_05933_gb300 import inputs
        probs = inputs.many_problems(args.many)
        mplan = vp.Plan.create_many([(p.src_xy, p.w, p.tgt_xy, p.csr, p.root) for p in probs], p_fmm=args.p,
                                    leaf=args.leaf, max_dens=1, flags=vp.VP_FLAG_GRAPH)
        mf = torch.as_tensor(np.concatenate([p.f for p in probs], axis=1), device=dev)
        mo = torch.empty((1, mplan.n_tgt), dtype=torch.float64, device=dev)
        movl = None
        if tuned is not None:
            from paper_2203_05933_gb300 import autotune
            movl = autotune.tune_overlap(mplan, mf, mo, choices=(0, 1, 2, 4, 8))
        mplan.eval(mf, out=mo)
        torch.cuda.synchronize()
        mt = timed(lambda: mplan.eval(mf, out=mo), max(3, args.steps // 3))
        mi = mplan.info()
        many = {"problems": len(probs), "n_tgt": int(mi.n_tgt), "nnz": int(mi.nnz), "levels": int(mi.n_levels),
                "value": mi.n_tgt / float(np.mean(mt)) / 1e6, "unit": UNIT, "ms_per_step": float(np.mean(mt)) * 1e3,
                "launches_per_eval": int(mi.last_launches), "graph": True, "overlap": movl}
        mplan.close()
        del mf, mo

    # oversampled leg: the same disk, densities at the p-nodes, FMM over the q = 2p nodes
    # (16 x 16 per box, 81 per triangle), same correction matrix
    upsampled = None
    if args.upsampled > 0 and rank == 0:
        from paper_2203_05933_gb300 import inputs
        t0 = time.perf_counter()
        uxy, uw, ups = inputs.disk_upsampling(seed=inputs.SEED_BASE + 2) if args.size == "full" else \
            inputs.disk_upsampling(base_level=5 if args.size == "small" else 6,
                                   fine_level=7 if args.size == "small" else 8, seed=inputs.SEED_BASE + 2)
        gen_s = time.perf_counter() - t0
        uplan = vp.Plan.create_upsampled(uxy, uw, prob.tgt_xy, prob.csr, ups, p_fmm=args.p, leaf=args.leaf,
                                         max_dens=1, flags=vp.VP_FLAG_GRAPH, root=prob.root)
        uo = torch.empty((1, prob.n_tgt), dtype=torch.float64, device=dev)
        for _ in range(max(3, args.warmup)):
            uplan.eval(f[:1], out=uo)
        torch.cuda.synchronize()
        ut = timed(lambda: uplan.eval(f[:1], out=uo), max(3, args.steps // 3))
        ui = uplan.info()
        upsampled = {"workload": prob.name + "_q2p", "n_q_nodes": int(ui.n_src), "n_f": int(ui.n_f),
                     "n_tgt": int(ui.n_tgt), "cells": int(ui.n_cells), "p2p_pairs": int(ui.p2p_pairs),
                     "value": prob.n_tgt / float(np.mean(ut)) / 1e6, "unit": UNIT,
                     "ms_per_step": float(np.mean(ut)) * 1e3, "input_gen_s": gen_s,
                     "launches_per_eval": int(ui.last_launches), "graph": True}
        uplan.close()
        del uo

    # interpolation leg: V from the disk's nodes to uniform random points of the disk
    interp_leg = None
    if args.interp > 0 and rank == 0:
        from paper_2203_05933_gb300 import inputs
        from paper_2203_05933_gb300.setup import interp as sinterp
        from paper_2203_05933_gb300.setup import meshes as smeshes
        base, fine = {"full": (7, 9), "medium": (6, 8), "small": (5, 7)}[args.size]
        t0 = time.perf_counter()
        mesh = smeshes.disk_mesh(base_level=base, fine_level=fine, centres=inputs.disk_centres(inputs.SEED_BASE + 2),
                                 refine_radius={base + 1: 0.11, base + 2: 0.04})
        rng = np.random.default_rng(21)
        rr = np.sqrt(rng.random(args.interp)) * (1.0 - 1e-9)
        th = rng.random(args.interp) * 2 * np.pi
        ipts = np.stack([rr * np.cos(th), rr * np.sin(th)], axis=1)
        icell, iref = sinterp.locate_mesh(mesh, ipts)
        gen_s = time.perf_counter() - t0
        ip = vp.Interp(sinterp.mesh_types(), np.where(mesh.cell_kind == 0, 0, 1).astype(np.int32), mesh.cell_start,
                       icell, iref)
        io = torch.empty((1, args.interp), dtype=torch.float64, device=dev)
        for _ in range(3):
            ip.eval(out[:1], out=io)
        torch.cuda.synchronize()
        it = timed(lambda: ip.eval(out[:1], out=io), max(3, args.steps // 3))
        interp_leg = {"points": args.interp, "node_values": prob.n_tgt, "cells": mesh.ncell,
                      "value": args.interp / float(np.mean(it)) / 1e6, "unit": "Mpoints/s",
                      "ms_per_step": float(np.mean(it)) * 1e3, "setup_s": gen_s,
                      "what": "V at uniform random points of the disk from V at the nodes "
                              "(per-cell coefficients + basis recurrences), launched on the evaluation stream"}
        ip.close()
        del io

    # triangle self-correction leg: the self blocks of every band triangle of the
    # disk generated on the GPU from the fixed reference-space rules
    tricorr_leg = None
    if args.tricorr > 0 and rank == 0:
        from paper_2203_05933_gb300 import inputs
        from paper_2203_05933_gb300.setup import meshes as smeshes
        from paper_2203_05933_gb300.setup import tricorr as stricorr
        base, fine = {"full": (7, 9), "medium": (6, 8), "small": (5, 7)}[args.size]
        t0 = time.perf_counter()
        rules = stricorr.self_rules(8)
        mesh = smeshes.disk_mesh(base_level=base, fine_level=fine, centres=inputs.disk_centres(inputs.SEED_BASE + 2),
                                 refine_radius={base + 1: 0.11, base + 2: 0.04})
        geom = np.array([stricorr.geom_params(g) for g in mesh.geom if g[0] == "tri"])
        setup_s = time.perf_counter() - t0
        tc = vp.TriCorr(rules)
        gdev = torch.as_tensor(geom, device=dev)
        tout = torch.empty((geom.shape[0], 36, 36), dtype=torch.float64, device=dev)
        tc.eval(gdev, out=tout)
        torch.cuda.synchronize()
        tt = timed(lambda: tc.eval(gdev, out=tout), 3)
        t0 = time.perf_counter()
        stricorr.self_corrections_reference([g for g in mesh.geom if g[0] == "tri"][0], rules)
        host_cell_s = time.perf_counter() - t0
        n_rule = int(rules["N"])
        flops = geom.shape[0] * 36 * (36 * n_rule * 2.0 + 36 * 36 * 2.0)
        ms = float(np.mean(tt)) * 1e3
        tricorr_leg = {"cells": int(geom.shape[0]), "targets_per_cell": 36, "rule_nodes_per_target": n_rule,
                       "ms": ms, "value": geom.shape[0] / (ms * 1e-3), "unit": "cells/s",
                       "contraction_tflops": flops / (ms * 1e-3) / 1e12, "fp64_peak_tflops": FP64_PEAK_TFLOPS,
                       "arith": "FP64 cell maps; mapped Green function and the 36 x rule-node contraction in "
                                "float-float (contraction_tflops counts its 2 flops per term)",
                       "host_numpy_s_per_cell": host_cell_s, "setup_s": setup_s}
        tc.close()

    # star leg: star with 12 holes, about 4.2 M sources and 2^22 targets (half nodes,
    # half random interior points), own-cell correction rows; same P and leaf
    star = None
    if args.star > 0 and rank == 0:
        from paper_2203_05933_gb300 import inputs
        t0 = time.perf_counter()
        sprob = inputs.star_problem("4M", csr="own")
        gen_s = time.perf_counter() - t0
        sp_, sl_, stune = args.p, args.leaf, None
        if tuned is not None:  # tune P and the leaf size on this geometry as well
            from paper_2203_05933_gb300 import autotune
            stune = autotune.tune(sprob.src_xy, sprob.w, sprob.tgt_xy, ndens=1, geometry=sprob.name,
                                  root=sprob.root, use_cache=False, steps=3, p_choices=(16, 24),
                                  leaf_choices=(64, 128))
            sp_, sl_ = stune["p_fmm"], stune["leaf"]
        t0 = time.perf_counter()
        splan = vp.Plan.create(sprob.src_xy, sprob.w, sprob.tgt_xy, sprob.csr, p_fmm=sp_, leaf=sl_,
                               max_dens=1, flags=vp.VP_FLAG_GRAPH, root=sprob.root)
        torch.cuda.synchronize()
        plan_s = time.perf_counter() - t0
        sf = torch.as_tensor(sprob.f, device=dev)
        so = torch.empty((1, sprob.n_tgt), dtype=torch.float64, device=dev)
        sovl = None
        if tuned is not None:
            sovl = autotune.tune_overlap(splan, sf, so, choices=(0, 1, 2, 4, 8))
        for _ in range(max(3, args.warmup)):
            splan.eval(sf, out=so)
        torch.cuda.synchronize()
        st = timed(lambda: splan.eval(sf, out=so), max(3, args.steps // 3))
        si = splan.info()
        star = {"workload": sprob.name, "n_src": sprob.n_src, "n_tgt": sprob.n_tgt, "nnz": sprob.nnz,
                "triangles": sprob.meta["n_triangles"], "p_fmm": int(si.p_fmm), "leaf": int(si.leaf),
                "p2p_pairs": int(si.p2p_pairs), "value": sprob.n_tgt / float(np.mean(st)) / 1e6, "unit": UNIT,
                "ms_per_step": float(np.mean(st)) * 1e3, "input_gen_s": gen_s, "plan_s": plan_s,
                "launches_per_eval": int(si.last_launches), "graph": True, "overlap": sovl,
                "autotune": None if stune is None else {
                    "table": [{k: r[k] for k in ("p_fmm", "leaf", "err", "ms")} for r in stune["table"]],
                    "tuning_s": stune["tuning_s"]}}
        splan.close()
        del sf, so, sprob

    # modified-Helmholtz leg: G = (lambda^2/2pi) K0(lambda r) on the same disk,
    # lambda^2 = 100 as in the paper's modified-Helmholtz experiment
    mh_leg = None
    if args.mhelm > 0 and rank == 0:
        lam = math.sqrt(args.mhelm)
        # (P, leaf) by time among the candidates whose result is within 1e-11 of the
        # P = 30 one (normalised by (lambda^2/2pi) sum |w f|), as the autotuner does
        cand = [(args.p, args.leaf)] if tuned is None else [(30, 64), (16, 64), (16, 128), (24, 64), (24, 128)]
        best, ref30, table = None, None, []
        scale = lam * lam / (2 * math.pi) * float(np.abs(prob.w * prob.f[0]).sum())
        for mp_, ml_ in cand:
            mplan_ = vp.Plan.create(prob.src_xy, prob.w, prob.tgt_xy, prob.csr, p_fmm=mp_, leaf=ml_,
                                    flags=vp.VP_FLAG_GRAPH, root=prob.root, kernel=vp.VP_KERNEL_MHELMHOLTZ,
                                    lam=lam)
            f1 = f[:1]
            o1 = torch.empty((1, prob.n_tgt), dtype=torch.float64, device=dev)
            for _ in range(2):
                mplan_.eval(f1, out=o1)
            torch.cuda.synchronize()
            tt = timed(lambda: mplan_.eval(f1, out=o1), 3)
            ms_ = float(np.mean(tt)) * 1e3
            if ref30 is None:
                ref30 = o1.clone()
            dev_err = float((o1 - ref30).abs().max()) / scale
            table.append({"p_fmm": mp_, "leaf": ml_, "ms": ms_, "err_vs_p30": dev_err})
            if dev_err <= 1e-11 and (best is None or ms_ < best[0]):
                if best is not None:
                    best[1].close()
                best = (ms_, mplan_, mp_, ml_)
            else:
                mplan_.close()
        del ref30
        _, mplan, mp_, ml_ = best
        f1 = f[:1]
        mo = torch.empty((1, prob.n_tgt), dtype=torch.float64, device=dev)
        movl = None
        if tuned is not None and prob.csr is not None:
            from paper_2203_05933_gb300 import autotune
            movl = autotune.tune_overlap(mplan, f1, mo, choices=(0, 2, 4))
        for _ in range(max(3, args.warmup)):
            mplan.eval(f1, out=mo)
        torch.cuda.synchronize()
        mt = timed(lambda: mplan.eval(f1, out=mo), max(3, args.steps // 3))
        mi = mplan.info()
        mo_host = mo.cpu().numpy()
        mplan.set_flags(vp.VP_FLAG_TIMING)
        mplan.eval(f1, out=mo)
        mph = mplan.phase_times()
        mplan.set_flags(vp.VP_FLAG_GRAPH)
        # near field in float-float on the FP32 pipes: the plan's modelled FP32
        # operation count (per evaluated distance 92 + 2 (deg - m + 1) + 24 m, +14 when
        # it serves both directions) against the FP32 issue rate; L2P and M2P (FP64)
        # run in the same kernel
        leaf_ms = mph.get("leaf", float("nan"))
        near_ops = int(mi.near_ops)
        mh_leg = {"workload": prob.name + f"_modified_helmholtz_lambda2_{args.mhelm:g}", "lambda": lam,
                  "p_fmm": int(mi.p_fmm), "leaf": int(mi.leaf), "n_tgt": prob.n_tgt,
                  "value": prob.n_tgt / float(np.mean(mt)) / 1e6, "unit": UNIT,
                  "ms_per_step": float(np.mean(mt)) * 1e3, "phase_ms": mph, "overlap": movl,
                  "launches_per_eval": int(mi.last_launches), "near_terms": int(mi.near_terms),
                  "p2p_pairs": int(mi.p2p_pairs), "graph": True,
                  "leaf_roofline": {"bound": "alu", "unit": "T FP32-ops/s", "peak": FP32_OPS_PEAK,
                                    "achieved": near_ops / (leaf_ms * 1e-3) / 1e12,
                                    "frac": near_ops / (leaf_ms * 1e-3) / 1e12 / FP32_OPS_PEAK,
                                    "per_unit": f"{near_ops / max(1, mi.p2p_evals):.0f} FP32 ops per evaluated "
                                                f"distance (plan model; {int(mi.p2p_evals)} evaluations for "
                                                f"{int(mi.p2p_pairs)} directed pairs)"},
                  "candidates": table}
        if not args.no_cpu:
            rec, err = cpu_baseline_mhelm(prob, lam, mo_host)
            mh_leg["cpu_baseline"] = rec
            mh_leg["rel_err"] = err
        mplan.close()

    if rank != 0:
        plan.close()
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    # roofline of the dominant phase, from live CUDA-event phase times on the evaluation stream
    models = roofline_models(info, prob)
    dom = max(phase_ms, key=phase_ms.get)
    rl_all = {}
    for name, m in models.items():
        ms = phase_ms.get(name)
        if not ms:
            continue
        scale = 1e9 if m["bound"] == "hbm" else 1e12
        achieved = m["work"] / (ms * 1e-3) / scale
        r = {"bound": m["bound"], "kernel": m["kernel"], "achieved": achieved, "peak": m["peak"],
             "unit": m["unit"], "frac": achieved / m["peak"], "traffic": None, "ms": ms,
             "peak_source": m["peak_source"], "per_unit": m["per_unit"]}
        if PROFILED_TRAFFIC.get(name) and m.get("units"):
            per, what, src = PROFILED_TRAFFIC[name]
            r["traffic"] = per * m["units"]
            r["traffic_source"] = f"ncu dram__bytes_read.sum + dram__bytes_write.sum per {what}, {src}, scaled"
        if "fp64_equiv_flop" in m:
            fe = m["fp64_equiv_flop"] / (ms * 1e-3) / 1e12
            r["fp64_equiv"] = {"achieved_tflops": fe, "fp64_peak_tflops": FP64_PEAK_TFLOPS,
                               "frac": fe / FP64_PEAK_TFLOPS}
        rl_all[name] = r
    roofline = dict(rl_all.get(dom, {}), phase=dom)
    cpu, rel_err = (None, None) if args.no_cpu else cpu_baseline(prob, out_first)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32x2", "data": "synthetic",
        "config": {"workload": prob.name, "n_src": prob.n_src, "n_tgt": prob.n_tgt, "nnz": prob.nnz,
                   "ndens": prob.ndens, "p_fmm": info.p_fmm, "leaf": info.leaf, "levels": info.n_levels,
                   "boxes": info.n_boxes, "p2p_pairs": info.p2p_pairs, "m2l_pairs": info.n_v_pairs,
                   "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replicas x{world}"},
        "rel_err": rel_err,
        "phase_ms": phase_ms,
        "roofline": roofline,
        "roofline_phases": rl_all,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(prob.ndens * prob.n_src * 8),
                "d2h_bytes_per_step": int(prob.ndens * prob.n_tgt * 8)},
        "batched": batched,
        "adjoint": adjoint,
        "many_problems": many,
        "star": star,
        "mhelm": mh_leg,
        "upsampled": upsampled,
        "interp": interp_leg,
        "tricorr": tricorr_leg,
        "clocks": clk,
        "gpu_launches": int(launches_per_eval * args.steps),
        "wall_s": wall,
        "graph": True,
        "overlap": overlap,
        "autotune": None if tuned is None else {
            "chosen": {"p_fmm": tuned["p_fmm"], "leaf": tuned["leaf"]}, "tol": tuned["tol"], "safety": tuned["safety"],
            "table": [{k: r[k] for k in ("p_fmm", "leaf", "err", "ms")} for r in tuned["table"]],
            "tuning_s": tuned["tuning_s"]},
    }
    print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
