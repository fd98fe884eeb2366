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


def test_static_exact_fill_and_split():
    # n_src + n_tgt equal to the scratch capacity: the source split must shrink
    # to one slice so that the charges and one row of partial sums fill it exactly
    n_src = 4097
    n_tgt = (1 << 21) - n_src
    rng = np.random.default_rng(11)
    src_np = rng.uniform(-1.0, 1.0, (n_src, 2))
    tgt_np = rng.uniform(-1.0, 1.0, (n_tgt, 2))
    tgt_np[:100] = src_np[:100]  # some coincident pairs
    w_np = rng.uniform(0.5, 1.5, n_src)
    f_np = rng.standard_normal((1, n_src))
    plan = vp.Plan.create(src_np, w_np, tgt_np, None, p_fmm=30, leaf=64, max_dens=1)
    src, tgt, w, f = _dev(src_np), _dev(tgt_np), _dev(w_np), _dev(f_np)
    nrm = float(np.abs(w_np * f_np[0]).sum())
    for call in range(2):
        ref = plan.eval(f).cpu().numpy()
        out = torch.full((1, n_tgt), np.nan, dtype=torch.float64, device="cuda")
        vp.vp_eval_direct_static(src, w, f, tgt, out)
        err = float(np.max(np.abs(out.cpu().numpy() - ref)) / nrm)
        assert err <= TOL, (call, err)
    plan.close()


def test_static_padded_leading_dimensions():
    # strided rows (ld = n + 7) and a source count that leaves a ragged last slice
    n_src, n_tgt, nd = 4096 * 3 + 1, 5000, 2
    rng = np.random.default_rng(12)
    src_np = rng.uniform(-1.0, 1.0, (n_src, 2))
    tgt_np = rng.uniform(-1.0, 1.0, (n_tgt, 2))
    w_np = rng.uniform(0.5, 1.5, n_src)
    f_np = rng.standard_normal((nd, n_src))
    fbuf = torch.full((nd, n_src + 7), np.nan, dtype=torch.float64, device="cuda")
    fbuf[:, :n_src] = _dev(f_np)
    obuf = torch.full((nd, n_tgt + 7), 123.0, dtype=torch.float64, device="cuda")
    plan = vp.Plan.create(src_np, w_np, tgt_np, None, p_fmm=30, leaf=64, max_dens=2)
    ref = plan.eval(_dev(f_np)).cpu().numpy()
    vp.vp_eval_direct_static(_dev(src_np), _dev(w_np), fbuf[:, :n_src], _dev(tgt_np), obuf[:, :n_tgt])
    got = obuf.cpu().numpy()
    nrm = np.abs(w_np[None, :] * f_np).sum(axis=1)[:, None]
    assert float(np.max(np.abs(got[:, :n_tgt] - ref) / nrm)) <= TOL
    assert np.all(got[:, n_tgt:] == 123.0)  # the padding is not written
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
