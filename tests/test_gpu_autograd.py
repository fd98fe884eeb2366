"""Differentiation through the autograd wrapper (adjoint and target gradients).

L = 0.5 ||V[f] - u*||^2 with seeded u*. dL/df (transposed FMM + transposed
correction) is checked against central finite differences along random
directions (exact up to rounding: L is quadratic in f) and against the
oracle's adjoint; dL/dt (differentiated expansions and direct sums, correction
held fixed) against the oracle's direct-sum gradient and against central
finite differences with h = 1e-6 at targets at least 1e-2 away from every
source (re-planning at the shifted targets).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2203_05933_gb300 import inputs, vp  # noqa: E402
from paper_2203_05933_gb300.autograd import volume_potential  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()
    oracle.build()


def _problem():
    p = inputs.cloud_problem(2500, 1200, ndens=2, shared=300, seed=51)
    return p


def test_grad_f_matches_finite_differences_and_oracle():
    p = _problem()
    plan = vp.Plan.create(p.src_xy, p.w, p.tgt_xy, p.csr, p_fmm=30, leaf=32, max_dens=2)
    rng = np.random.default_rng(8)
    ustar = torch.as_tensor(rng.standard_normal((2, p.n_tgt)), device="cuda")
    f = torch.as_tensor(p.f, device="cuda").requires_grad_(True)
    V = volume_potential(plan, f)
    L = 0.5 * ((V - ustar) ** 2).sum()
    L.backward()
    g = f.grad.detach()
    # oracle adjoint applied to the residual
    resid = (V.detach() - ustar).cpu().numpy()
    ref = oracle.adjoint(p.src_xy, p.w, resid, p.tgt_xy, p.csr)
    scale = np.abs(resid).sum(axis=1)[:, None] * p.w.max()
    assert np.max(np.abs(g.cpu().numpy() - ref) / scale) <= 1e-10
    # central differences along random directions (L quadratic in f)
    for k in range(3):
        dirn = torch.as_tensor(rng.standard_normal(p.f.shape), device="cuda")
        h = 1e-3
        with torch.no_grad():
            Lp = 0.5 * ((plan.eval(f.detach() + h * dirn) - ustar) ** 2).sum()
            Lm = 0.5 * ((plan.eval(f.detach() - h * dirn) - ustar) ** 2).sum()
        fd = float((Lp - Lm) / (2 * h))
        an = float((g * dirn).sum())
        assert abs(fd - an) <= 1e-8 * max(1.0, abs(an)), (fd, an)
    plan.close()


def test_grad_targets_matches_oracle_and_finite_differences():
    p = _problem()
    # targets away from every source for the finite-difference part
    d = np.hypot(*(p.tgt_xy[:, None, :] - p.src_xy[None, :, :]).transpose(2, 0, 1)).min(axis=1)
    plan = vp.Plan.create(p.src_xy, p.w, p.tgt_xy, p.csr, p_fmm=30, leaf=32, max_dens=2)
    rng = np.random.default_rng(9)
    ustar = torch.as_tensor(rng.standard_normal((2, p.n_tgt)), device="cuda")
    f = torch.as_tensor(p.f, device="cuda")
    t = torch.as_tensor(p.tgt_xy, device="cuda").requires_grad_(True)
    V = volume_potential(plan, f, t)
    L = 0.5 * ((V - ustar) ** 2).sum()
    L.backward()
    gt = t.grad.cpu().numpy()
    resid = (V.detach() - ustar).cpu().numpy()
    ref = oracle.grad_targets(p.src_xy, p.w, p.f, resid, p.tgt_xy)
    scale = oracle.grad_scale(p.src_xy, p.w, p.f, resid, p.tgt_xy)
    assert np.max(np.abs(gt - ref) / scale[:, None]) <= 1e-10
    # finite differences on a few far-from-source targets, correction held fixed
    far = np.nonzero(d > 1e-2)[0][:4]
    h = 1e-6
    for i in far:
        for k in range(2):
            vals = []
            for sgn in (1, -1):
                tt = p.tgt_xy.copy()
                tt[i, k] += sgn * h
                pl = vp.Plan.create(p.src_xy, p.w, tt, p.csr, p_fmm=30, leaf=32, max_dens=2,
                                    root=(-1.0, -1.0, 2.0))
                with torch.no_grad():
                    vals.append(float(0.5 * ((pl.eval(f) - ustar) ** 2).sum()))
                pl.close()
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - gt[i, k]) <= 1e-5 * max(1.0, abs(gt[i, k])), (i, k, fd, gt[i, k])
    plan.close()
