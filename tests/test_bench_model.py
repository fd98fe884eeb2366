"""The benchmark's roofline bookkeeping (bench.roofline_of), on a stand-in of the
plan statistics of the 4 M star: each phase is reported against the bound its
kernel has (HBM for the correction product, the FP64 FMA peak for the others),
achieved = the algorithmic work of one launch over its time, frac = achieved
over the peak, and the DRAM traffic scaled from the profiled bytes per unit."""

import types

import pytest

bench = pytest.importorskip("bench")


def _info():
    return types.SimpleNamespace(n_tgt=4194304, n_src=4169056, nnz=2391975976, n_v_pairs=5067680,
                                 p2p_pairs=1263948433, p2p_evals=1263948433, p_fmm=24, leaf=64, sym_slots=0)


def test_phases_and_bounds():
    info = _info()
    ms = {"leaf": 11.23, "m2l": 5.46, "out": 3.20, "upward": 1.02, "l2l": 0.46}
    r = bench.roofline_of(ms, info, 1, 1.25, "stand-in")
    assert set(r) == {"leaf", "m2l", "out", "upward"}
    # the correction product: HBM, algorithmic bytes over the time
    out = r["out"]
    assert out["bound"] == "hbm" and out["unit"] == "GB/s"
    gbs = (info.nnz * 8.0 + info.n_tgt * 8.0 * 3) / (3.20e-3) / 1e9
    assert out["achieved"] == pytest.approx(gbs)
    assert out["frac"] == pytest.approx(gbs / out["peak"])
    assert out["traffic"] == pytest.approx(bench.PROFILED_TRAFFIC["out"][0] * info.nnz)
    # the FP64 phases: flops by the survey's accounting over the FP64 FMA peak
    leaf = r["leaf"]
    assert leaf["bound"] == "alu" and leaf["unit"] == "TFLOP/s" and leaf["peak"] == 1.25
    flop = info.p2p_pairs * bench.P2P_FLOP_PER_PAIR + info.n_tgt * 8.0 * 24
    assert leaf["achieved"] == pytest.approx(flop / 11.23e-3 / 1e12)
    assert leaf["frac"] == pytest.approx(leaf["achieved"] / 1.25)
    assert leaf["traffic"] == pytest.approx(bench.PROFILED_TRAFFIC["leaf"][0] * info.n_tgt)
    m2l = r["m2l"]
    assert m2l["achieved"] == pytest.approx(info.n_v_pairs * 8.0 * 25 ** 2 / 5.46e-3 / 1e12)
    assert m2l["pipe_ops_tops"] == pytest.approx(info.n_v_pairs * bench.F64_OPS_M2L_PER_P * 24 / 5.46e-3 / 1e12)
    up = r["upward"]
    assert up["achieved"] == pytest.approx(info.n_src * 8.0 * 24 / 1.02e-3 / 1e12)


def test_traffic_only_for_the_profiled_configuration():
    # the profiled bytes per unit hold for P = 24 and one density; other
    # configurations report traffic null
    info = _info()
    info.p_fmm = 16
    r = bench.roofline_of({"leaf": 5.0, "out": 3.0}, info, 1, 1.25, "stand-in")
    assert r["leaf"]["traffic"] is None and r["out"]["traffic"] is None
    r = bench.roofline_of({"leaf": 5.0}, _info(), 8, 1.25, "stand-in")
    assert r["leaf"]["traffic"] is None
