"""Interpolation set-up (host): the simplex basis equals the formula the C ABI
states (scaled Legendre times Jacobi, checked against scipy's special
functions), values-to-coefficients maps invert their Vandermonde matrices,
point location inverts the cell maps, and the interpolant reproduces
polynomials exactly on boxes and straight triangles."""

import numpy as np
from scipy.special import eval_jacobi, eval_legendre

from paper_2203_05933_gb300.setup import interp, meshes, simplex


def test_simplex_basis_matches_stated_formula():
    rng = np.random.default_rng(1)
    u = rng.random((400, 2))
    u = u[u.sum(axis=1) < 0.999]
    xi, eta = u[:, 0], u[:, 1]
    V = simplex.orthogonal_basis(xi, eta, 7)
    s, t, b = 2 * xi - 1 + eta, 1 - eta, 2 * eta - 1
    col = 0
    for m in range(8):
        for k in range(8 - m):
            ref = eval_legendre(m, s / t) * t**m * eval_jacobi(k, 2 * m + 1, 0, b)
            assert np.max(np.abs(V[:, col] - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))
            col += 1
    assert col == V.shape[1] == 36


def test_coefficient_maps_invert_vandermonde():
    t, _ = np.polynomial.legendre.leggauss(8)
    X, Y = np.meshgrid(t, t, indexing="xy")
    Vb = interp.legendre2_basis(X.ravel(), Y.ravel(), 8)
    assert np.max(np.abs(interp.box_coef(8) @ Vb - np.eye(64))) < 1e-12
    xi, eta, _ = simplex.simplex_rule(8)
    Vt = simplex.orthogonal_basis(xi, eta, 7)
    assert np.max(np.abs(interp.simplex_coef(8) @ Vt - np.eye(36))) < 1e-9


def test_locate_inverts_maps_and_interpolant_reproduces_polynomials():
    m = meshes.disk_mesh(base_level=3, fine_level=4, centres=[[0.3, -0.2]], refine_radius={4: 0.3})
    rng = np.random.default_rng(2)
    r = np.sqrt(rng.random(1500)) * 0.9999
    th = rng.random(1500) * 2 * np.pi
    pts = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    cell, ref = interp.locate_mesh(m, pts)
    for k in range(0, 1500, 7):
        g = m.geom[cell[k]]
        if g[0] == "box":
            x = g[1] + g[3] / 2 * (1 + ref[k, 0])
            y = g[2] + g[3] / 2 * (1 + ref[k, 1])
        else:
            xy = (simplex.affine_map(g[1], ref[k:k + 1, 0], ref[k:k + 1, 1])[0] if g[2] is None else
                  simplex.blended_map(g[1], g[2], ref[k:k + 1, 0], ref[k:k + 1, 1])[0])
            x, y = xy[0]
        assert abs(x - pts[k, 0]) + abs(y - pts[k, 1]) < 1e-13
    ct = np.where(m.cell_kind == 0, 0, 1)
    types = interp.mesh_types()
    f = lambda x, y: x**3 * y**2 - 2 * y**5 + x  # noqa: E731  (total degree 5)
    V = interp.interpolate_reference(types, ct, m.cell_start, f(m.xy[:, 0], m.xy[:, 1]), cell, ref)[0]
    exact = f(pts[:, 0], pts[:, 1])
    kind = m.cell_kind[cell]
    assert np.max(np.abs(V - exact)[kind < 2]) < 1e-13
    assert np.max(np.abs(V - exact)[kind == 2]) < 1e-6  # curved: the map is not polynomial
