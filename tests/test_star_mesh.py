"""The star-with-holes workload (r(theta) = 1 + 0.3 cos 5 theta, 12 circular
holes): its cells form a quadrature rule for the domain, checked against
polynomial moments computed independently (spectrally accurate periodic
trapezoid sums over the boundary curves), and its targets and correction
pattern follow their stated recipe."""

import math

import numpy as np
import pytest

from paper_2203_05933_gb300 import inputs
from paper_2203_05933_gb300.setup import meshes


def _moment_star(a, b, n_theta=4096):
    # int_star x^a y^b dA = int_0^2pi r(theta)^(a+b+2) / (a+b+2) cos^a sin^b dtheta
    th = 2 * math.pi * np.arange(n_theta) / n_theta
    r = 1.0 + 0.3 * np.cos(5 * th)
    return float(np.sum(r ** (a + b + 2) / (a + b + 2) * np.cos(th) ** a * np.sin(th) ** b) * 2 * math.pi / n_theta)


def _moment_disk(cx, cy, R, a, b, n_phi=256, n_rho=16):
    t, wt = np.polynomial.legendre.leggauss(n_rho)
    rho = R * (t + 1) / 2
    wr = wt * R / 2
    phi = 2 * math.pi * np.arange(n_phi) / n_phi
    P, F = np.meshgrid(rho, phi, indexing="ij")
    val = (cx + P * np.cos(F)) ** a * (cy + P * np.sin(F)) ** b * P
    return float(np.sum(val * wr[:, None]) * 2 * math.pi / n_phi)


@pytest.fixture(scope="module")
def star_small():
    holes, _, _, _ = inputs.star_geometry()
    return holes, meshes.star_mesh(holes, base_level=7, fine_level=7)


def test_star_mesh_integrates_polynomials(star_small):
    holes, m = star_small
    assert np.all(m.w > 0)
    for a, b in [(0, 0), (2, 0), (1, 1), (0, 3), (4, 2), (3, 4)]:
        exact = _moment_star(a, b) - sum(_moment_disk(cx, cy, R, a, b) for cx, cy, R in holes)
        got = float(np.sum(m.w * m.xy[:, 0] ** a * m.xy[:, 1] ** b))
        assert abs(got - exact) <= 1e-12 * max(1.0, abs(exact)), (a, b, got, exact)
    assert abs(m.area - _moment_star(0, 0) + sum(math.pi * R * R for _, _, R in holes)) < 1e-13


def test_star_mesh_nodes_lie_inside_and_cells_are_consistent(star_small):
    holes, m = star_small
    assert np.all(meshes.inside_star(m.xy[:, 0], m.xy[:, 1], holes))
    assert m.cell_start[-1] == m.n
    # every triangle band cell has 36 nodes, every box 64
    sizes = np.diff(m.cell_start)
    assert np.all(sizes[m.cell_kind == 0] == 64) and np.all(sizes[m.cell_kind > 0] == 36)
    # curved triangles on the outer curve and on each hole
    assert (m.cell_kind == 2).sum() > 12 * 8


def test_holes_respect_the_gaps():
    holes, cen, width, amp = inputs.star_geometry()
    assert holes.shape == (12, 3) and np.all((holes[:, 2] >= 0.02) & (holes[:, 2] <= 0.08))
    for i in range(12):
        for j in range(i):
            d = math.hypot(holes[i, 0] - holes[j, 0], holes[i, 1] - holes[j, 1])
            assert d - holes[i, 2] - holes[j, 2] >= 0.12
    th = np.linspace(0, 2 * math.pi, 20000, endpoint=False)
    r = 1 + 0.3 * np.cos(5 * th)
    bnd = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    for cx, cy, R in holes:
        assert np.min(np.hypot(bnd[:, 0] - cx, bnd[:, 1] - cy)) - R >= 0.12 - 1e-9
    assert cen.shape == (50, 2) and np.all((width >= 1e-3) & (width <= 1e-1))
    assert np.all(meshes.inside_star(cen[:, 0], cen[:, 1], holes))


def test_star_small_problem_targets_and_pattern():
    p = inputs.star_problem("small", csr="own")
    assert p.n_tgt == 1 << 14
    holes = p.meta["holes"]
    assert np.all(meshes.inside_star(p.tgt_xy[:, 0], p.tgt_xy[:, 1], holes))
    # the first half are nodes (exact copies), the rest random interior points
    n_sub = p.n_tgt // 2
    src = {tuple(x) for x in p.src_xy}
    assert all(tuple(x) in src for x in p.tgt_xy[:n_sub:97])
    rowptr, col, val = p.csr
    assert rowptr.size == p.n_tgt + 1 and np.all(np.diff(rowptr) > 0)
    # own-cell rows: contiguous node ranges of one cell, a node row holds the node itself
    for i in range(0, n_sub, 211):
        c = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(c) == 1)
        j = np.nonzero((p.src_xy[:, 0] == p.tgt_xy[i, 0]) & (p.src_xy[:, 1] == p.tgt_xy[i, 1]))[0]
        assert j.size == 1 and c[0] <= j[0] <= c[-1]


def test_cell_rows_csr_matches_a_loop():
    cs = np.array([0, 3, 7, 9], np.int64)
    tc = np.array([2, 0, 1, 1, 2])
    rowptr, col = inputs.cell_rows_csr(cs, tc)
    ref = np.concatenate([np.arange(cs[c], cs[c + 1]) for c in tc])
    assert np.array_equal(col, ref) and np.array_equal(np.diff(rowptr), np.diff(cs)[tc])
    cols = [np.array([5, 1], np.int32), np.array([0], np.int32), np.array([2, 3, 4], np.int32)]
    rowptr, col = inputs.cell_rows_csr(cs, tc, cols)
    assert np.array_equal(col, np.concatenate([cols[c] for c in tc]))
