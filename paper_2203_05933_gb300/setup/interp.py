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


def _invert_triangle(v, curve, p, iters: int = 40):
    """Reference coordinates of the points p [k, 2] in one triangle (affine, or
    blended when curve is given: Newton from the affine guess). Returns
    (ref [k, 2], converged [k])."""
    p = np.atleast_2d(p)
    A = np.array([[v[1, 0] - v[0, 0], v[2, 0] - v[0, 0]], [v[1, 1] - v[0, 1], v[2, 1] - v[0, 1]]])
    r = np.linalg.solve(A, (p - v[0]).T).T
    if curve is None:
        return r, np.ones(p.shape[0], bool)
    xi, eta = r[:, 0].copy(), r[:, 1].copy()
    for _ in range(iters):
        xi = np.clip(xi, 0.0, 1.0 - 1e-12)
        x, y, xx, yx, xe, ye = simplex.blended_map_jacobian(v, curve, xi, eta)
        rx, ry = x - p[:, 0], y - p[:, 1]
        det = xx * ye - xe * yx
        dxi = (ye * rx - xe * ry) / det
        deta = (-yx * rx + xx * ry) / det
        xi, eta = xi - dxi, eta - deta
        if np.max(np.abs(dxi) + np.abs(deta)) < 1e-15:
            break
    x, y, *_ = simplex.blended_map_jacobian(v, curve, np.clip(xi, 0.0, 1.0 - 1e-12), eta)
    ok = np.abs(x - p[:, 0]) + np.abs(y - p[:, 1]) < 1e-12
    return np.stack([xi, eta], axis=1), ok


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
    tris = np.array([k for k, g in enumerate(mesh.geom) if g[0] == "tri"], np.int64)
    todo = np.nonzero(cell < 0)[0]
    if todo.size and tris.size:
        from scipy.spatial import cKDTree

        cen = np.array([mesh.geom[k][1].mean(axis=0) for k in tris])
        kk = min(8, tris.size)
        _, cand = cKDTree(cen).query(pts[todo], k=kk)
        cand = cand.reshape(todo.size, kk)
        for j in range(kk):
            left = cell[todo] < 0
            if not left.any():
                break
            idx = todo[left]
            cj = cand[left, j]
            for c in np.unique(cj):
                sel = idx[cj == c]
                k = int(tris[c])
                _, v, curve = mesh.geom[k]
                r, ok = _invert_triangle(v, curve, pts[sel])
                inside = ok & (r[:, 0] >= -1e-10) & (r[:, 1] >= -1e-10) & (r[:, 0] + r[:, 1] <= 1 + 1e-10)
                cell[sel[inside]] = k
                ref[sel[inside]] = r[inside]
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
