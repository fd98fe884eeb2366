"""The allocation-free entry point against the planned evaluation.

vp_eval_direct_static exists for callers that cannot allocate device memory
when they evaluate (their host owns every allocation, or an allocation would
break a stream capture they are inside). It keeps its scratch in a fixed
device array, so this test checks that two calls in a row (the second one
reusing the array the first one left behind) both agree with vp_eval on a plan
to the tolerance of the other parity tests. The file name makes pytest collect
it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05933_gb300 import inputs, vp  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


@pytest.mark.parametrize("case", ["boxgrid", "cloud"])
def test_static_matches_planned_eval_twice(case):
    if case == "boxgrid":
        prob = inputs.box_grid_problem(nbox=6, order=8, ndens=2)
    else:
        prob = inputs.cloud_problem(3000, 2500, ndens=3, shared=500, seed=31)
    plan = vp.Plan.create(prob.src_xy, prob.w, prob.tgt_xy, prob.csr, p_fmm=30, leaf=32, max_dens=4,
                          root=prob.root)
    scale = inputs.normaliser(prob)[:, None]
    src, tgt, w = _dev(prob.src_xy), _dev(prob.tgt_xy), _dev(prob.w)
    csr = (_dev(prob.csr[0], torch.int64), _dev(prob.csr[1], torch.int32), _dev(prob.csr[2]))
    rng = np.random.default_rng(7)
    for call in range(2):
        fnp = prob.f if call == 0 else rng.standard_normal(prob.f.shape)
        f = _dev(fnp)
        ref = plan.eval(f).cpu().numpy()
        out = torch.full((prob.ndens, prob.n_tgt), np.nan, dtype=torch.float64, device="cuda")
        vp.vp_eval_direct_static(src, w, f, tgt, out, csr)
        got = out.cpu().numpy()
        nrm = np.abs(prob.w[None, :] * fnp).sum(axis=1)[:, None] if call else scale
        err = float(np.max(np.abs(got - ref) / nrm))
        assert np.all(np.isfinite(got)) and err <= TOL, (call, err)
    plan.close()


def test_static_rejects_oversize():
    n = (1 << 21) // 2 + 1  # n_src + n_tgt above the scratch capacity
    src = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(vp.VPError) as ei:
        vp.vp_eval_direct_static(src, w, f, src, out)
    assert ei.value.status == 1
