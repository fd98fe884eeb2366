"""The star-with-holes workloads on the GPU, checked on sampled outputs
against the CPU oracle.

4M case: about 4.17 M quadrature sources, 2^22 targets (a seeded half of the
nodes plus uniform random interior points), own-cell correction rows, in the
benchmark's launch configuration (P = 16, leaf 128).

1M differentiation case: about 0.97 M sources, targets = the nodes plus the
centres of the larger holes, self + near correction rows;
L = 0.5 ||V[f] - u*||^2 with seeded u*. dL/df through the adjoint against the
oracle's transposed sum on sampled sources and against central differences
along random directions (L is quadratic in f, so the difference quotient is
exact up to rounding for any step); dL/dt against the oracle's direct-sum
gradient on a 16 384-target subsample and against central differences with
h = 1e-6 at the hole centres (at least 0.03 from every source).
"""

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2203_05933_gb300 import inputs, vp  # noqa: E402
from paper_2203_05933_gb300.autograd import volume_potential  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()
    oracle.build()


def test_star_4M_sampled_targets():
    prob = inputs.star_problem("4M", csr="own")
    plan = vp.Plan.create(prob.src_xy, prob.w, prob.tgt_xy, prob.csr, root=prob.root, p_fmm=16, leaf=128,
                          max_dens=1)
    out = plan.eval(torch.as_tensor(prob.f, device="cuda")).cpu().numpy()
    plan.close()
    n_sub = min(prob.n_src // 2, prob.n_tgt // 2)  # node targets come first
    rng = np.random.default_rng(11)
    # node targets, random interior targets, and the last target (ragged end)
    rows = np.unique(np.concatenate([rng.choice(n_sub, 96, replace=False),
                                     n_sub + rng.choice(prob.n_tgt - n_sub, 96, replace=False),
                                     [prob.n_tgt - 1]]))
    ref = oracle.evaluate(prob.src_xy, prob.w, prob.f, prob.tgt_xy[rows], oracle.csr_rows(prob.csr, rows))
    err = float(np.max(np.abs(out[:, rows] - ref) / inputs.normaliser(prob)[:, None]))
    print(f"star 4M ({prob.n_src} sources, {prob.n_tgt} targets) sampled rel err {err:.3e}")
    assert err <= TOL


def _csr_cols(csr, cols):
    rowptr, col, val = csr
    n_rows = rowptr.size - 1
    m = sp.csr_matrix((val, col, rowptr), shape=(n_rows, int(col.max()) + 1))[:, cols].tocsr()
    m.sort_indices()
    return m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64)


def test_star_1M_differentiation():
    holes, _, _, _ = inputs.star_geometry()
    centres = holes[holes[:, 2] >= 0.03][:, :2]
    prob = inputs.star_problem("1M", targets="nodes", csr="near", extra_targets=centres)
    n_ex = centres.shape[0]
    plan = vp.Plan.create(prob.src_xy, prob.w, prob.tgt_xy, prob.csr, root=prob.root, p_fmm=30, leaf=64,
                          max_dens=1)
    rng = np.random.default_rng(12)
    ustar = torch.as_tensor(rng.standard_normal((1, prob.n_tgt)), device="cuda")
    f = torch.as_tensor(prob.f, device="cuda").requires_grad_(True)
    t = torch.as_tensor(prob.tgt_xy, device="cuda").requires_grad_(True)
    V = volume_potential(plan, f, t)
    L = 0.5 * ((V - ustar) ** 2).sum()
    L.backward()
    gf = f.grad.detach()
    gt = t.grad.cpu().numpy()
    resid = (V.detach() - ustar).cpu().numpy()

    # dL/df: oracle transposed sum on sampled sources
    cols = np.sort(rng.choice(prob.n_src, 256, replace=False))
    ref = oracle.adjoint(prob.src_xy[cols], prob.w[cols], resid, prob.tgt_xy, _csr_cols(prob.csr, cols))
    scale = np.abs(resid).sum() * prob.w.max()
    err_f = float(np.max(np.abs(gf.cpu().numpy()[:, cols] - ref)) / scale)
    print(f"star 1M dL/df rel err {err_f:.3e}")
    assert err_f <= TOL
    # central differences along random directions
    for h in (1e-3, 1e-6):
        dirn = torch.as_tensor(rng.standard_normal(prob.f.shape), device="cuda")
        with torch.no_grad():
            Lp = float(0.5 * ((plan.eval(f.detach() + h * dirn) - ustar) ** 2).sum())
            Lm = float(0.5 * ((plan.eval(f.detach() - h * dirn) - ustar) ** 2).sum())
        fd = (Lp - Lm) / (2 * h)
        an = float((gf * dirn).sum())
        # rounding of L (about 1e-16 |L|) divided by 2h bounds the quotient's error
        tol = 1e-8 * abs(an) + 4e-16 * abs(Lp) / h
        print(f"  h={h:g} fd {fd:.12e} adjoint {an:.12e}")
        assert abs(fd - an) <= tol, (h, fd, an)
    plan.close()

    # dL/dt: oracle direct-sum gradient on a 16k subsample (the hole centres included)
    rows = np.unique(np.concatenate([rng.choice(prob.n_tgt - n_ex, 16384 - n_ex, replace=False),
                                     np.arange(prob.n_tgt - n_ex, prob.n_tgt)]))
    ref_t = oracle.grad_targets(prob.src_xy, prob.w, prob.f, resid[:, rows], prob.tgt_xy[rows])
    scale_t = oracle.grad_scale(prob.src_xy, prob.w, prob.f, resid[:, rows], prob.tgt_xy[rows])
    err_t = float(np.max(np.abs(gt[rows] - ref_t) / scale_t[:, None]))
    err_m = float(np.max(np.abs(gt[rows] - ref_t)) / np.max(np.abs(ref_t)))
    print(f"star 1M dL/dt rel err {err_t:.3e} per target (sum of |terms|), {err_m:.3e} of max |ref|, "
          f"on {rows.size} targets")
    assert err_t <= TOL

    # central differences of V at the hole centres, h = 1e-6 (one plan holds every shifted point)
    h = 1e-6
    shifts = []
    for c in centres:
        for k in range(2):
            for sgn in (1.0, -1.0):
                p = c.copy()
                p[k] += sgn * h
                shifts.append(p)
    shifts = np.array(shifts)
    fd_plan = vp.Plan.create(prob.src_xy, prob.w, shifts, None, root=prob.root, p_fmm=30, leaf=64, max_dens=1)
    with torch.no_grad():
        vs = fd_plan.eval(f.detach()).cpu().numpy()[0]
    fd_plan.close()
    for i in range(n_ex):
        for k in range(2):
            dV = (vs[4 * i + 2 * k] - vs[4 * i + 2 * k + 1]) / (2 * h)
            want = gt[prob.n_tgt - n_ex + i, k]
            got = resid[0, prob.n_tgt - n_ex + i] * dV
            assert abs(got - want) <= 1e-5 * max(1.0, abs(want)), (i, k, got, want)
