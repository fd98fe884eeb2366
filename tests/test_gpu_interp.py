"""Interpolation of nodal values to arbitrary points on the GPU
(vp_interp_create / vp_interp_eval) against the plain definition
basis(ref) @ C @ v (setup.interp.interpolate_reference), exact polynomial
reproduction, and the off-node volume potential obtained by interpolating
vp_eval's nodal output."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2203_05933_gb300 import inputs, vp  # noqa: E402
from paper_2203_05933_gb300.setup import corrections as C  # noqa: E402
from paper_2203_05933_gb300.setup import interp, meshes  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()
    oracle.build()


def _disk_points(m, n, seed):
    rng = np.random.default_rng(seed)
    r = np.sqrt(rng.random(n)) * 0.9999
    th = rng.random(n) * 2 * np.pi
    pts = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    return pts, *interp.locate_mesh(m, pts)


def test_disk_interpolation_matches_definition():
    m = meshes.disk_mesh(base_level=4, fine_level=5, centres=[[0.2, 0.1]], refine_radius={5: 0.25})
    pts, cell, ref = _disk_points(m, 5000, 3)
    types = interp.mesh_types()
    ct = np.where(m.cell_kind == 0, 0, 1).astype(np.int32)
    ip = vp.Interp(types, ct, m.cell_start, cell, ref)
    v = np.random.default_rng(4).standard_normal((3, m.n))
    out = ip.eval(torch.as_tensor(v, device="cuda")).cpu().numpy()
    want = interp.interpolate_reference(types, ct, m.cell_start, v, cell, ref)
    err = float(np.max(np.abs(out - want)) / np.max(np.abs(want)))
    print(f"interpolation rel err {err:.2e} ({np.bincount(m.cell_kind[cell])} points per cell kind)")
    assert err < 1e-13
    # polynomial of total degree 6: exact on boxes and straight triangles
    f = lambda x, y: x**4 * y**2 - 3 * x * y**5 + y  # noqa: E731
    vp_ = ip.eval(torch.as_tensor(f(m.xy[:, 0], m.xy[:, 1]), device="cuda")).cpu().numpy()
    kind = m.cell_kind[cell]
    assert np.max(np.abs(vp_ - f(pts[:, 0], pts[:, 1]))[kind < 2]) < 1e-13
    ip.close()


def test_off_node_potential_by_interpolation():
    # V at the nodes (GPU FMM + area-to-line corrections), interpolated to
    # random points, against V evaluated directly at those points by the oracle
    # with the corrections of those points
    nbox = 6
    p = inputs.box_grid_problem(nbox=nbox, order=8, csr="corrections")
    plan = vp.Plan.create(p.src_xy, p.w, p.tgt_xy, p.csr, p_fmm=30, leaf=64, root=(-1.0, -1.0, 2.0))
    Vn = plan.eval(torch.as_tensor(p.f, device="cuda"))
    plan.close()
    rng = np.random.default_rng(5)
    pts = rng.uniform(-0.999, 0.999, size=(300, 2))
    side = 2.0 / nbox
    bx = np.minimum(((pts[:, 0] + 1) // side).astype(int), nbox - 1)
    by = np.minimum(((pts[:, 1] + 1) // side).astype(int), nbox - 1)
    cell = (by * nbox + bx).astype(np.int32)
    ref = np.stack([(pts[:, 0] + 1 - (bx + 0.5) * side) / (side / 2), (pts[:, 1] + 1 - (by + 0.5) * side) / (side / 2)],
                   axis=1)
    ip = vp.Interp([(interp.BASIS_LEGENDRE2, 8, interp.box_coef(8))], np.zeros(nbox * nbox, np.int32),
                   np.arange(nbox * nbox + 1) * 64, cell, ref)
    Vi = ip.eval(Vn).cpu().numpy()
    ip.close()
    Vd = oracle.evaluate(p.src_xy, p.w, p.f, pts, C.box_grid_corrections_at(pts, nbox, 8))
    err = float(np.max(np.abs(Vi - Vd)) / np.max(np.abs(Vd)))
    print(f"off-node potential: interpolated vs direct rel diff {err:.2e}")
    assert err < 1e-6


def test_interp_bad_arguments_raise():
    types = [(interp.BASIS_LEGENDRE2, 8, interp.box_coef(8))]
    with pytest.raises(vp.VPError):
        vp.Interp(types, np.zeros(2, np.int32), np.array([0, 64, 127]), np.zeros(1, np.int32), np.zeros((1, 2)))
    with pytest.raises(vp.VPError):
        vp.Interp(types, np.zeros(2, np.int32), np.array([0, 64, 128]), np.array([2], np.int32), np.zeros((1, 2)))
    with pytest.raises(vp.VPError):
        vp.Interp([(interp.BASIS_SIMPLEX, 8, interp.box_coef(8))], np.zeros(1, np.int32), np.array([0, 64]),
                  np.zeros(1, np.int32), np.zeros((1, 2)))
