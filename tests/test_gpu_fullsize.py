"""The benchmark's full-size workloads in the launch configuration bench.py
times (P = 16, leaf 128, graph replay), checked on sampled outputs against the
CPU oracle: one density (symmetric near field), a pass of 8 densities, the
adjoint, and the oversampled (q = 2p) form of the same disk."""

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2203_05933_gb300 import inputs, vp  # noqa: E402
from paper_2203_05933_gb300.setup import upsample as U  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def disk():
    return inputs.disk_problem(seed=inputs.SEED_BASE + 2, name="disk_1M")


def test_disk_1M_bench_configuration(disk):
    prob = disk
    plan = vp.Plan.create(prob.src_xy, prob.w, prob.tgt_xy, prob.csr, p_fmm=16, leaf=128, max_dens=8,
                          flags=vp.VP_FLAG_GRAPH, root=prob.root)
    assert plan.info().sym_slots > 0
    rng = np.random.default_rng(31)
    rows = rng.choice(prob.n_tgt, size=128, replace=False)
    # one density
    f1 = torch.as_tensor(prob.f, device="cuda")
    out1 = plan.eval(f1).cpu().numpy()
    ref1 = oracle.evaluate(prob.src_xy, prob.w, prob.f, prob.tgt_xy[rows], oracle.csr_rows(prob.csr, rows))
    e1 = float(np.max(np.abs(out1[:, rows] - ref1) / inputs.normaliser(prob)[:, None]))
    # a pass of 8 seeded random densities (the batched leg's chunk)
    f8 = rng.standard_normal((8, prob.n_src))
    out8 = plan.eval(torch.as_tensor(f8, device="cuda")).cpu().numpy()
    ref8 = oracle.evaluate(prob.src_xy, prob.w, f8[:, :], prob.tgt_xy[rows[:32]], oracle.csr_rows(prob.csr, rows[:32]))
    norm8 = np.abs(prob.w[None, :] * f8).sum(axis=1)[:, None]
    e8 = float(np.max(np.abs(out8[:, rows[:32]] - ref8) / norm8))
    # the adjoint on sampled sources
    g = rng.standard_normal((1, prob.n_tgt))
    gf, _ = plan.adjoint(torch.as_tensor(g, device="cuda"))
    cols = np.sort(rng.choice(prob.n_src, size=64, replace=False))
    M = sp.csr_matrix((prob.csr[2], prob.csr[1], prob.csr[0]), shape=(prob.n_tgt, prob.n_src))[:, cols].tocsr()
    ref_a = oracle.adjoint(prob.src_xy[cols], prob.w[cols], g, prob.tgt_xy,
                           (M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data))
    ea = float(np.max(np.abs(gf.cpu().numpy()[:, cols] - ref_a)) / (np.abs(g).sum() * prob.w.max()))
    plan.close()
    print(f"disk 1M P=16 leaf 128: one density {e1:.2e}, 8 densities {e8:.2e}, adjoint {ea:.2e}")
    assert e1 <= TOL and e8 <= TOL and ea <= TOL


def test_disk_1M_oversampled(disk):
    prob = disk
    xq, wq, ups = inputs.disk_upsampling(seed=inputs.SEED_BASE + 2)
    plan = vp.Plan.create_upsampled(xq, wq, prob.tgt_xy, prob.csr, ups, p_fmm=16, leaf=128, max_dens=1,
                                    flags=vp.VP_FLAG_GRAPH, root=prob.root)
    out = plan.eval(torch.as_tensor(prob.f, device="cuda")).cpu().numpy()
    plan.close()
    rows = np.random.default_rng(32).choice(prob.n_tgt, size=64, replace=False)
    fq = U.apply(ups, prob.f)
    ref = oracle.evaluate(xq, wq, fq, prob.tgt_xy[rows], None)
    M = sp.csr_matrix((prob.csr[2], prob.csr[1], prob.csr[0]), shape=(prob.n_tgt, prob.n_src))
    ref = ref + (M[rows] @ prob.f.T).T
    err = float(np.max(np.abs(out[:, rows] - ref)) / np.abs(fq * wq[None, :]).sum())
    print(f"oversampled disk ({xq.shape[0]} q-nodes) sampled rel err {err:.2e}")
    assert err <= TOL
