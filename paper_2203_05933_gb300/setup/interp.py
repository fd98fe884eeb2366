"""Set-up for interpolating nodal values to arbitrary points (Sec. 3.2.1,
Eq. vals_to_coeffs; Sec. 4.2): the values-to-coefficients maps of the cell
types, and the location of points in cells with their reference coordinates
(inverse cell maps; Newton's method for the blended maps of curved
triangles). Host work, done once for static geometry; the evaluation itself
runs in libvp (vp_interp_create / vp_interp_eval).

Basis conventions are the ones the C ABI states:
  boxes      P_i(xi) P_j(eta) on [-1, 1]^2, index j * order + i;
  triangles  setup.simplex.orthogonal_basis of total degree order - 1.
"""

from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre

from . import simplex

BASIS_LEGENDRE2 = 0
BASIS_SIMPLEX = 1


def legendre2_basis(xi, eta, order: int) -> np.ndarray:
    """[npts, order^2] values of P_i(xi) P_j(eta), column j * order + i."""
    xi = np.asarray(xi, float)
    eta = np.asarray(eta, float)
    Px = np.stack([eval_legendre(i, xi) for i in range(order)], axis=1)
    Py = np.stack([eval_legendre(j, eta) for j in range(order)], axis=1)
    return (Py[:, :, None] * Px[:, None, :]).reshape(xi.size, order * order)


def box_coef(order: int = 8) -> np.ndarray:
    """C = V^-1 for the order x order Gauss-Legendre box nodes (y-major, x fastest)."""
    t, _ = np.polynomial.legendre.leggauss(order)
    X, Y = np.meshgrid(t, t, indexing="xy")
    return np.linalg.inv(legendre2_basis(X.ravel(), Y.ravel(), order))


def simplex_coef(p: int = 8) -> np.ndarray:
    """C = V^-1 for the p(p+1)/2 simplex nodes of setup.simplex (degree p - 1)."""
    xi, eta, _ = simplex.simplex_rule(p)
    return np.linalg.inv(simplex.orthogonal_basis(xi, eta, p - 1))


def mesh_types(box_order: int = 8, tri_p: int = 8):
    """[(basis, order, C)] for boxes (type 0) and triangles (type 1)."""
    return [(BASIS_LEGENDRE2, box_order, box_coef(box_order)), (BASIS_SIMPLEX, tri_p, simplex_coef(tri_p))]


def _invert_triangle(v, curve, p, iters: int = 30):
    """Reference coordinates of point p in the triangle (affine, or blended when
    curve is given); Newton from the affine guess for curved triangles."""
    A = np.array([[v[1, 0] - v[0, 0], v[2, 0] - v[0, 0]], [v[1, 1] - v[0, 1], v[2, 1] - v[0, 1]]])
    r = np.linalg.solve(A, p - v[0])
    if curve is None:
        return r, True
    xi, eta = float(r[0]), float(r[1])
    for _ in range(iters):
        xi_c = min(max(xi, 0.0), 1.0 - 1e-12)
        x, y, xx, yx, xe, ye = simplex.blended_map_jacobian(v, curve, np.array([xi_c]), np.array([eta]))
        res = np.array([x[0] - p[0], y[0] - p[1]])
        J = np.array([[xx[0], xe[0]], [yx[0], ye[0]]])
        step = np.linalg.solve(J, res)
        xi, eta = xi_c - step[0], eta - step[1]
        if np.max(np.abs(step)) < 1e-15:
            break
    x, y, *_ = simplex.blended_map_jacobian(v, curve, np.array([min(max(xi, 0.0), 1.0 - 1e-12)]), np.array([eta]))
    ok = abs(x[0] - p[0]) + abs(y[0] - p[1]) < 1e-12
    return np.array([xi, eta]), ok


def locate_mesh(mesh, pts, tol: float = 1e-12):
    """Cell and reference coordinates of every point (inside the meshed domain).
    Boxes by a per-level hash of integer box coordinates; the rest by bounding
    boxes and the inverse triangle maps. Returns (cell int32 [n], ref [n, 2])."""
    pts = np.asarray(pts, float).reshape(-1, 2)
    n = pts.shape[0]
    cell = np.full(n, -1, np.int64)
    ref = np.zeros((n, 2))
    boxes = [(k, g[1], g[2], g[3]) for k, g in enumerate(mesh.geom) if g[0] == "box"]
    if boxes:
        side = np.array([b[3] for b in boxes])
        for s in np.unique(side):
            sel = [b for b in boxes if b[3] == s]
            ids = np.array([b[0] for b in sel])
            x0 = min(b[1] for b in boxes) - 4 * side.max()
            y0 = min(b[2] for b in boxes) - 4 * side.max()
            ix = np.round((np.array([b[1] for b in sel]) - x0) / s).astype(np.int64)
            iy = np.round((np.array([b[2] for b in sel]) - y0) / s).astype(np.int64)
            key = iy * (1 << 31) + ix
            order = np.argsort(key)
            key, ids_s = key[order], ids[order]
            todo = np.nonzero(cell < 0)[0]
            px = np.floor((pts[todo, 0] - x0) / s).astype(np.int64)
            py = np.floor((pts[todo, 1] - y0) / s).astype(np.int64)
            q = py * (1 << 31) + px
            pos = np.clip(np.searchsorted(key, q), 0, key.size - 1)
            hit = key[pos] == q
            hp = todo[hit]
            cid = ids_s[pos[hit]]
            cell[hp] = cid
            g = [mesh.geom[c] for c in cid]
            cx = np.array([gg[1] + gg[3] / 2 for gg in g]) if g else np.zeros(0)
            cy = np.array([gg[2] + gg[3] / 2 for gg in g]) if g else np.zeros(0)
            ref[hp, 0] = (pts[hp, 0] - cx) / (s / 2)
            ref[hp, 1] = (pts[hp, 1] - cy) / (s / 2)
    tris = [k for k, g in enumerate(mesh.geom) if g[0] == "tri"]
    todo = np.nonzero(cell < 0)[0]
    if todo.size and tris:
        bb = mesh.cell_bbox[tris]
        for i in todo:
            p = pts[i]
            cand = np.nonzero((bb[:, 0] - tol <= p[0]) & (p[0] <= bb[:, 1] + tol) & (bb[:, 2] - tol <= p[1])
                              & (p[1] <= bb[:, 3] + tol))[0]
            for c in cand:
                k = tris[c]
                _, v, curve = mesh.geom[k]
                r, ok = _invert_triangle(v, curve, p)
                if ok and r[0] >= -1e-10 and r[1] >= -1e-10 and r[0] + r[1] <= 1 + 1e-10:
                    cell[i] = k
                    ref[i] = r
                    break
    if np.any(cell < 0):
        raise ValueError(f"{int(np.sum(cell < 0))} points lie in no cell")
    return cell.astype(np.int32), ref


def interpolate_reference(mesh_types_, cell_type, node_start, values, cell, ref) -> np.ndarray:
    """Plain evaluation of the definition, for checks: for each point,
    basis(ref) @ C @ values[cell nodes]."""
    values = np.atleast_2d(values)
    out = np.empty((values.shape[0], cell.size))
    for k in range(cell.size):
        c = cell[k]
        basis, order, C = mesh_types_[cell_type[c]]
        v = values[:, node_start[c]:node_start[c + 1]]
        if basis == BASIS_LEGENDRE2:
            phi = legendre2_basis(ref[k:k + 1, 0], ref[k:k + 1, 1], order)[0]
        else:
            phi = simplex.orthogonal_basis(ref[k:k + 1, 0], ref[k:k + 1, 1], order - 1)[0]
        out[:, k] = (v @ C.T) @ phi
    return out
