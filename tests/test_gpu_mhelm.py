"""Parity of the modified-Helmholtz path (VP_KERNEL_MHELMHOLTZ, through the C
ABI) with the CPU oracle oracle/mhelm.py.

Kernel G = (lambda^2/2pi) K0(lambda r) (arXiv 2203.05933, Sec. 2). Error metric:
max |V_gpu - V_oracle| / ((lambda^2/2pi) sum_j |w_j f_j|), the Laplace metric
with the kernel's prefactor; the bar is 1e-10. Adjoint: the same with
max_j w_j sum_i |g_i| in place of sum_j |w_j f_j|.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mhelm  # noqa: E402
from paper_2203_05933_gb300 import inputs, vp  # noqa: E402

TOL = 1e-10
MH = vp.VP_KERNEL_MHELMHOLTZ


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()


def norm(prob, lam):
    return lam * lam / (2 * math.pi) * inputs.normaliser(prob)


def make(prob, lam, **opts):
    return vp.Plan.create(prob.src_xy, prob.w, prob.tgt_xy, prob.csr, root=prob.root, kernel=MH, lam=lam, **opts)


@pytest.mark.parametrize("lam,P", [(1.0, 30), (3.0, 24), (10.0, 24), (10.0, 30), (60.0, 24)])
def test_cloud_matches_oracle(lam, P):
    # adaptive cloud with V, W and X lists; 1500 targets coincide with sources;
    # at lambda = 60 many near-field pairs have lambda r > 2 (integral path of K0).
    # (P = 16 truncates at about 1e-9 on this clustered cloud for every lambda.)
    prob = inputs.cloud_problem(6000, 5000, ndens=1, shared=1500, seed=71)
    plan = make(prob, lam, p_fmm=P, leaf=32)
    info = plan.info()
    assert info.n_x_pairs > 0 and info.n_w_pairs > 0 and info.n_v_pairs > 0
    out = plan.eval(torch.as_tensor(prob.f, device="cuda")).cpu().numpy()
    ref = mhelm.evaluate(prob.src_xy, prob.w, prob.f, prob.tgt_xy, lam, prob.csr)
    err = float(np.max(np.abs(out - ref) / norm(prob, lam)[:, None]))
    print(f"modified Helmholtz lambda={lam} P={P}: rel err {err:.2e}")
    assert err <= TOL
    plan.close()


@pytest.mark.parametrize("lam", [2.0, 10.0, 60.0])
def test_float_float_near_field_matches_fp64(lam):
    # the float-float near field (VP_FLAG_FF: FP32 pipes, FP32 series tails)
    # against the all-FP64 one (the default), same P and tree
    prob = inputs.cloud_problem(6000, 5000, ndens=1, shared=1500, seed=77)
    f = torch.as_tensor(prob.f, device="cuda")
    res = {}
    for flags in (vp.VP_FLAG_FF, 0):
        plan = make(prob, lam, p_fmm=24, leaf=64, flags=flags)
        res[flags] = plan.eval(f).cpu().numpy()
        plan.close()
    err = float(np.max(np.abs(res[vp.VP_FLAG_FF] - res[0]) / norm(prob, lam)[:, None]))
    print(f"modified Helmholtz lambda={lam}: float-float vs FP64 near field {err:.2e}")
    assert err <= 1e-12


def test_symmetric_near_field_matches_fp64():
    # targets = nodes: each distance between adjacent leaves is evaluated once for
    # both directions (slots + reduction); against the all-FP64 directed near field
    prob = inputs.disk_problem(base_level=5, fine_level=6)
    lam = 10.0
    f = torch.as_tensor(prob.f, device="cuda")
    res = {}
    for flags in (vp.VP_FLAG_FF, 0):
        plan = make(prob, lam, p_fmm=24, leaf=64, flags=flags)
        info = plan.info()
        assert (info.sym_slots > 0) == (flags == vp.VP_FLAG_FF)
        res[flags] = plan.eval(f).cpu().numpy()
        plan.close()
    err = float(np.max(np.abs(res[vp.VP_FLAG_FF] - res[0]) / norm(prob, lam)[:, None]))
    print(f"modified Helmholtz symmetric vs FP64 near field {err:.2e}")
    assert err <= 1e-12


def test_densities_graph_and_timing():
    # several densities (one pass each), graph replay bitwise equal to the plain
    # launch sequence, phase timing names
    prob = inputs.cloud_problem(3000, 2500, ndens=3, shared=500, seed=72)
    lam = 5.0
    f = torch.as_tensor(prob.f, device="cuda")
    plain = make(prob, lam, p_fmm=24, leaf=48)
    a = plain.eval(f).cpu().numpy()
    ref = mhelm.evaluate(prob.src_xy, prob.w, prob.f, prob.tgt_xy, lam, prob.csr)
    assert float(np.max(np.abs(a - ref) / norm(prob, lam)[:, None])) <= TOL
    graph = make(prob, lam, p_fmm=24, leaf=48, flags=vp.VP_FLAG_GRAPH)
    b1 = graph.eval(f).cpu().numpy()
    b2 = graph.eval(f).cpu().numpy()
    assert np.array_equal(a, b1) and np.array_equal(b1, b2)
    assert graph.info().last_launches > 0
    plain.set_flags(vp.VP_FLAG_TIMING)
    plain.eval(f)
    names = list(plain.phase_times())
    for want in ("charges", "upward", "m2l", "l2l", "leaf", "out"):
        assert want in names
    plain.close()
    graph.close()


def test_adjoint_matches_oracle():
    prob = inputs.cloud_problem(4000, 3500, ndens=2, shared=800, seed=73)
    lam = 8.0
    g = np.random.default_rng(4).standard_normal((2, prob.n_tgt))
    plan = make(prob, lam, p_fmm=24, leaf=40)
    gf = plan.adjoint(torch.as_tensor(g, device="cuda"))[0].cpu().numpy()
    ref = mhelm.adjoint(prob.src_xy, prob.w, g, prob.tgt_xy, lam, prob.csr)
    scale = lam * lam / (2 * math.pi) * prob.w.max() * np.abs(g).sum(axis=1)
    err = float(np.max(np.abs(gf - ref) / scale[:, None]))
    print(f"modified Helmholtz adjoint rel err {err:.2e}")
    assert err <= TOL
    with pytest.raises(vp.VPError):
        plan.adjoint(torch.as_tensor(g, device="cuda"), f=torch.as_tensor(prob.f, device="cuda"), grad_tgt=True)
    plan.close()


def test_adjoint_symmetric_near_field():
    # node targets: the transposed pass of the float-float kernels also takes the
    # symmetric near field
    prob = inputs.disk_problem(base_level=5, fine_level=6, ndens=2)
    lam = 10.0
    g = np.random.default_rng(6).standard_normal((2, prob.n_tgt))
    plan = make(prob, lam, p_fmm=24, leaf=64, flags=vp.VP_FLAG_FF)
    assert plan.info().sym_slots > 0
    gf = plan.adjoint(torch.as_tensor(g, device="cuda"))[0].cpu().numpy()
    sub = np.random.default_rng(7).choice(prob.n_src, size=300, replace=False)
    ref = mhelm.adjoint_cols(prob.src_xy, prob.w, g, prob.tgt_xy, sub, lam, prob.csr)
    scale = lam * lam / (2 * math.pi) * prob.w.max() * np.abs(g).sum(axis=1)
    err = float(np.max(np.abs(gf[:, sub] - ref) / scale[:, None]))
    print(f"modified Helmholtz adjoint (symmetric near field) rel err {err:.2e}")
    assert err <= TOL
    plan.close()


def test_disk_sampled_targets():
    # the paper's modified-Helmholtz experiment is on the unit disk with lambda^2 = 100
    prob = inputs.disk_problem(base_level=5, fine_level=7)
    lam = 10.0
    plan = make(prob, lam, p_fmm=16, leaf=128)  # 4e-11 on this geometry
    out = plan.eval(torch.as_tensor(prob.f, device="cuda")).cpu().numpy()
    rows = np.random.default_rng(9).choice(prob.n_tgt, size=300, replace=False)
    ref = mhelm.evaluate_rows(prob.src_xy, prob.w, prob.f, prob.tgt_xy, rows, lam, prob.csr)
    err = float(np.max(np.abs(out[:, rows] - ref) / norm(prob, lam)[:, None]))
    print(f"disk {prob.n_tgt} nodes, lambda=10: rel err {err:.2e}")
    assert err <= TOL
    plan.close()


def test_box_grid():
    prob = inputs.box_grid_problem(nbox=6, order=8)
    lam = 10.0
    plan = make(prob, lam, p_fmm=30, leaf=64)
    out = plan.eval(torch.as_tensor(prob.f, device="cuda")).cpu().numpy()
    ref = mhelm.evaluate(prob.src_xy, prob.w, prob.f, prob.tgt_xy, lam, prob.csr)
    assert float(np.max(np.abs(out - ref) / norm(prob, lam)[:, None])) <= TOL
    plan.close()


def test_edge_cases():
    lam = 3.0
    # one source, the target on it: nothing but the correction
    src = np.array([[0.25, -0.5]])
    w = np.array([2.0])
    plan = vp.Plan.create(src, w, src.copy(), None, kernel=MH, lam=lam)
    out = plan.eval(torch.ones((1, 1), dtype=torch.float64, device="cuda")).cpu().numpy()
    assert out[0, 0] == 0.0
    plan.close()
    # ragged sizes, no correction
    prob = inputs.cloud_problem(37, 1, ndens=1, seed=74, csr_per_row=0)
    plan = make(prob, lam, p_fmm=24, leaf=8)
    out = plan.eval(torch.as_tensor(prob.f, device="cuda")).cpu().numpy()
    ref = mhelm.evaluate(prob.src_xy, prob.w, prob.f, prob.tgt_xy, lam)
    assert float(np.max(np.abs(out - ref) / norm(prob, lam)[:, None])) <= TOL
    plan.close()
    # no targets
    prob = inputs.cloud_problem(50, 10, ndens=1, seed=75, csr_per_row=0)
    plan = vp.Plan.create(prob.src_xy, prob.w, np.zeros((0, 2)), None, kernel=MH, lam=lam)
    assert plan.eval(torch.as_tensor(prob.f, device="cuda")).shape[1] == 0
    plan.close()


def test_rejected_options():
    prob = inputs.cloud_problem(500, 400, ndens=1, seed=76, csr_per_row=0)
    with pytest.raises(vp.VPError):  # lambda must be > 0
        make(prob, 0.0)
    with pytest.raises(vp.VPError):  # expansion tables out of range
        make(prob, 1e-12, p_fmm=30, leaf=8)
