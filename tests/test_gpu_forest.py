"""The 256-problem batch (uneven square and disk problems of 2k-64k points in
one forest plan, one CUDA graph per evaluation) against the oracle: sampled
rows of every problem, each checked against that problem alone (interactions
never cross problems), forward and adjoint, float64 and float-float."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2203_05933_gb300 import inputs, vp  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()
    oracle.build()


def _csr_cols(csr, cols):
    """The CSR restricted to the given columns (renumbered 0..len(cols)-1)."""
    import scipy.sparse as sp

    rowptr, col, val = csr
    m = sp.csr_matrix((val, col, rowptr), shape=(rowptr.size - 1, int(col.max()) + 1))[:, cols].tocsr()
    m.sort_indices()
    return m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64)


@pytest.fixture(scope="module")
def forest():
    return inputs.many_problems(256)


@pytest.mark.parametrize("flags", [0, vp.VP_FLAG_FF])
def test_256_problems_sampled_rows(forest, flags):
    probs = forest
    plan = vp.Plan.create_many([(p.src_xy, p.w, p.tgt_xy, p.csr, p.root) for p in probs], p_fmm=16, leaf=64,
                               max_dens=1, flags=vp.VP_FLAG_GRAPH | flags)
    info = plan.info()
    assert info.n_problems == 256
    f = torch.as_tensor(np.concatenate([p.f for p in probs], axis=1), device="cuda")
    out = plan.eval(f).cpu().numpy()[0]
    rng = np.random.default_rng(31)
    g = rng.standard_normal((1, plan.n_tgt))
    gf = plan.adjoint(torch.as_tensor(g, device="cuda"))[0].cpu().numpy()[0]
    worst, worst_a, col = 0.0, 0.0, 0
    for k, p in enumerate(probs):
        rows = np.sort(rng.choice(p.n_tgt, size=min(12, p.n_tgt), replace=False))
        ref = oracle.evaluate(p.src_xy, p.w, p.f, p.tgt_xy[rows], oracle.csr_rows(p.csr, rows))[0]
        err = float(np.max(np.abs(out[col + rows] - ref)) / np.abs(p.w * p.f[0]).sum())
        worst = max(worst, err)
        # adjoint on sampled sources: the transposed sum (charges g at this problem's
        # targets, nodes = targets here) plus Pi^T g
        gk = g[:, col:col + p.n_tgt]
        ref_a = oracle.adjoint(p.src_xy[rows], p.w[rows], gk, p.tgt_xy, _csr_cols(p.csr, rows))[0]
        err_a = float(np.max(np.abs(gf[col + rows] - ref_a)) / (np.abs(gk).sum() * p.w.max()))
        worst_a = max(worst_a, err_a)
        col += p.n_tgt
    print(f"256 problems ({info.n_tgt} targets, flags={flags}): forward {worst:.2e}, adjoint {worst_a:.2e}")
    assert worst <= TOL and worst_a <= TOL
    plan.close()
