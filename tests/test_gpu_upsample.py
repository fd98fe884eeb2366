"""Oversampled smooth quadrature on the GPU (vp_plan_create_upsampled) against
the CPU oracle: the oracle interpolates f to the q-nodes cell by cell with the
same set-up matrices (plain dense products), sums directly over the q-nodes
and applies the correction to the p-node values; the adjoint and the target
gradient follow the same definition."""

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2203_05933_gb300 import inputs, vp  # noqa: E402
from paper_2203_05933_gb300.setup import corrections as C  # noqa: E402
from paper_2203_05933_gb300.setup import meshes  # noqa: E402
from paper_2203_05933_gb300.setup import upsample as U  # noqa: E402

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()
    oracle.build()


def _oracle_forward(xq, wq, ups, f, tgt, csr):
    V = oracle.evaluate(xq, wq, U.apply(ups, f), tgt, None)
    if csr is not None:
        M = sp.csr_matrix((csr[2], csr[1], csr[0]), shape=(tgt.shape[0], ups.n_f))
        V = V + (M @ f.T).T
    return V


def _oracle_adjoint(xq, wq, ups, g, tgt, csr):
    u = oracle.adjoint(xq, wq, g, tgt, None)  # w_j sum_i G(r_j, t_i) g_i at the q-nodes
    out = np.zeros((g.shape[0], ups.n_f))
    mats = [ups.dense(t) for t in range(len(ups.types))]
    for k in range(ups.cell_type.size):
        O = mats[ups.cell_type[k]]
        out[:, ups.f_start[k]:ups.f_start[k + 1]] = u[:, ups.src_start[k]:ups.src_start[k + 1]] @ O
    if csr is not None:
        M = sp.csr_matrix((csr[2], csr[1], csr[0]), shape=(tgt.shape[0], ups.n_f))
        out += (M.T @ g.T).T
    return out


def _disk_upsampled(base=4, fine=6, ndens=3, seed=77):
    cen = inputs.disk_centres(seed)
    rr = {base + 1: 0.2, base + 2: 0.08}
    mp = meshes.disk_mesh(base_level=base, fine_level=fine, centres=cen, refine_radius=rr)
    rule = U.collapsed_triangle_rule(9)
    mq = meshes.disk_mesh(base_level=base, fine_level=fine, centres=cen, refine_radius=rr, box_order=16,
                          tri_rule=rule)
    ups = U.mesh_upsampling(mp, mq, 8, 16, 8, rule)
    rowptr, col = meshes.near_cell_pattern(mp)
    csr = (rowptr, col, inputs.synthetic_csr_values(rowptr, col, mp.w, seed + 1))
    rng = np.random.default_rng(seed + 2)
    f = rng.standard_normal((ndens, mp.n)) + 1.0
    return mp, mq, ups, csr, f


@pytest.mark.parametrize("flags", [0, vp.VP_FLAG_FF, vp.VP_FLAG_FP64])
def test_box_grid_upsampled_constant_density_is_exact(flags):
    nbox = 6
    p = inputs.box_grid_problem(nbox=nbox, order=8, csr="none")
    xq, wq, ups = U.box_grid_upsampled(nbox, 8, 16)
    csr = C.box_grid_csr(nbox, 8, q=16)
    plan = vp.Plan.create_upsampled(xq, wq, p.tgt_xy, csr, ups, p_fmm=30, leaf=64, max_dens=2, flags=flags,
                                    root=(-1.0, -1.0, 2.0))
    assert plan.n_f == p.n_src and plan.n_src == xq.shape[0]
    import __graft_entry__ as ge
    exact = ge.ref_square(p.tgt_xy)
    v1 = plan.eval(torch.ones((1, p.n_src), dtype=torch.float64, device="cuda")).cpu().numpy()[0]
    err1 = float(np.max(np.abs(v1 - exact)))
    print(f"upsampled box grid f=1 abs err {err1:.2e}")
    assert err1 <= 1e-12
    f = np.random.default_rng(5).standard_normal((2, p.n_src))
    out = plan.eval(torch.as_tensor(f, device="cuda")).cpu().numpy()
    ref = _oracle_forward(xq, wq, ups, f, p.tgt_xy, csr)
    norm = np.abs(U.apply(ups, f) * wq[None, :]).sum(axis=1)
    assert float(np.max(np.abs(out - ref) / norm[:, None])) <= TOL
    plan.close()


@pytest.mark.parametrize("flags", [0, vp.VP_FLAG_FF, vp.VP_FLAG_FP64])
def test_disk_upsampled_forward_adjoint_gradient(flags):
    mp, mq, ups, csr, f = _disk_upsampled()
    tgt = mp.xy  # the p-nodes are the targets
    plan = vp.Plan.create_upsampled(mq.xy, mq.w, tgt, csr, ups, p_fmm=30, leaf=64, max_dens=2, flags=flags,
                                    root=(-1.0, -1.0, 2.0))
    info = plan.info()
    assert info.n_cells == mp.ncell and info.n_f == mp.n
    out = plan.eval(torch.as_tensor(f, device="cuda")).cpu().numpy()
    ref = _oracle_forward(mq.xy, mq.w, ups, f, tgt, csr)
    norm = np.abs(U.apply(ups, f) * mq.w[None, :]).sum(axis=1)
    err = float(np.max(np.abs(out - ref) / norm[:, None]))
    print(f"upsampled disk ({mq.n} q-nodes, {mp.n} p-nodes) rel err {err:.3e}")
    assert err <= TOL
    # adjoint (three densities: chunks of 2 and 1)
    g = np.random.default_rng(3).standard_normal((3, tgt.shape[0]))
    gf, _ = plan.adjoint(torch.as_tensor(g, device="cuda"))
    ref_a = _oracle_adjoint(mq.xy, mq.w, ups, g, tgt, csr)
    # scale: sum_i |g_i| times the largest sum_j |O_ji| w_j (the transposed sum's bound per unit kernel)
    mats = [np.abs(ups.dense(t)) for t in range(len(ups.types))]
    colw = max(float(np.max(mq.w[ups.src_start[k]:ups.src_start[k + 1]] @ mats[ups.cell_type[k]]))
               for k in range(ups.cell_type.size))
    scale = np.abs(g).sum(axis=1)[:, None] * colw
    err_a = float(np.max(np.abs(gf.cpu().numpy() - ref_a) / scale))
    print(f"upsampled adjoint rel err {err_a:.3e}")
    assert err_a <= TOL
    # dot-product identity <A f, g> = <f, A^T g>
    lhs = float(np.sum(out[:2] * g[:2]))
    rhs = float(np.sum(f[:2] * gf.cpu().numpy()[:2]))
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + np.abs(g[:2]).sum() * norm[:2].max())
    # target gradient (correction held fixed)
    _, gt = plan.adjoint(torch.as_tensor(g[:2], device="cuda"), grad_f=False, f=torch.as_tensor(f[:2], device="cuda"),
                         grad_tgt=True)
    ref_t = oracle.grad_targets(mq.xy, mq.w, U.apply(ups, f[:2]), g[:2], tgt)
    scale_t = oracle.grad_scale(mq.xy, mq.w, U.apply(ups, f[:2]), g[:2], tgt)
    err_t = float(np.max(np.abs(gt.cpu().numpy() - ref_t) / scale_t[:, None]))
    print(f"upsampled target gradient rel err {err_t:.3e}")
    assert err_t <= TOL
    plan.close()


def test_upsampled_host_entry_point_and_graph():
    mp, mq, ups, csr, f = _disk_upsampled(base=3, fine=5, ndens=1, seed=78)
    plan = vp.Plan.create_upsampled(mq.xy, mq.w, mp.xy, csr, ups, p_fmm=24, leaf=64, max_dens=1,
                                    flags=vp.VP_FLAG_GRAPH, root=(-1.0, -1.0, 2.0))
    fd = torch.as_tensor(f, device="cuda")
    a = plan.eval(fd).cpu().numpy()
    b = plan.eval(fd).cpu().numpy()  # graph replay
    c = plan.eval_host(f)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    plan.close()


def test_upsampled_bad_descriptions_raise():
    xq, wq, ups = U.box_grid_upsampled(2, 8, 16)
    tgt = inputs.box_grid_problem(nbox=2, order=8, csr="none").tgt_xy
    bad = U.Upsampling(types=ups.types, cell_type=ups.cell_type.copy(), f_start=ups.f_start.copy(),
                       src_start=ups.src_start.copy())
    bad.cell_type[1] = 3  # type out of range
    with pytest.raises(vp.VPError):
        vp.Plan.create_upsampled(xq, wq, tgt, None, bad)
    bad = U.Upsampling(types=ups.types, cell_type=ups.cell_type, f_start=ups.f_start.copy(),
                       src_start=ups.src_start.copy())
    bad.f_start[2] += 1  # count differs from the type
    with pytest.raises(vp.VPError):
        vp.Plan.create_upsampled(xq, wq, tgt, None, bad)
    with pytest.raises(vp.VPError):  # cells do not cover the sources
        vp.Plan.create_upsampled(np.vstack([xq, [[0.1, 0.2]]]), np.append(wq, 1.0), tgt, None, ups)
    rp = np.arange(tgt.shape[0] + 1, dtype=np.int64)
    col = np.full(tgt.shape[0], ups.n_f, np.int32)  # column past the p-nodes
    with pytest.raises(vp.VPError):
        vp.Plan.create_upsampled(xq, wq, tgt, (rp, col, np.ones(tgt.shape[0])), ups)
