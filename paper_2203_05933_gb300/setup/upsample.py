"""Oversampled smooth quadrature (Sec. 2, "Oversampled smooth quadratures";
Remark after Eq. nsrcs; Sec. 4.2 for boxes): the density is sampled at the
p-nodes of each cell, interpolated to the nodes of a finer smooth rule of order
q by a fixed per-cell-type matrix O_{p,q}, and the FMM sums over the q-nodes
with their weights (Jacobians folded in):

    V_k[f](r0) ~ sum_j G(R_k(xi_j, eta_j), r0) (O_{p,q} f_p^k)_j J_k(xi_j, eta_j) w_j .

Boxes: p x p tensor Gauss-Legendre nodes interpolated to q x q tensor
Gauss-Legendre nodes; O is the Kronecker product of two 1-D Lagrange
interpolation matrices (rows and columns ordered y-major, x fastest, as the
box generators order nodes). Triangles: the p(p+1)/2 simplex nodes of
setup.simplex interpolated (orthonormal basis of total degree < p,
O = V_q C_p with C_p the values-to-coefficients map, Eq. vals_to_coeffs) to a
collapsed Gauss rule with m^2 nodes, exact for total degree 2m - 2 (a stand-in
for the order-q Vioreanu-Rokhlin rule, which is not available here).

Host set-up only (untimed); the matrices are inputs of the evaluation.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import simplex


def lagrange_matrix(x_from: np.ndarray, x_to: np.ndarray) -> np.ndarray:
    """L[r, i] = l_i(x_to[r]) for the Lagrange basis on the nodes x_from
    (barycentric form, Berrut and Trefethen 2004)."""
    x_from = np.asarray(x_from, float)
    x_to = np.asarray(x_to, float)
    n = x_from.size
    wb = np.array([1.0 / np.prod([x_from[i] - x_from[k] for k in range(n) if k != i]) for i in range(n)])
    L = np.empty((x_to.size, n))
    for r, x in enumerate(x_to):
        d = x - x_from
        hit = np.nonzero(d == 0.0)[0]
        if hit.size:
            L[r] = 0.0
            L[r, hit[0]] = 1.0
            continue
        t = wb / d
        L[r] = t / t.sum()
    return L


def box_upsample_1d(p: int, q: int) -> np.ndarray:
    """1-D interpolation from p to q Gauss-Legendre nodes on [-1, 1]: [q, p]."""
    xp, _ = np.polynomial.legendre.leggauss(p)
    xq, _ = np.polynomial.legendre.leggauss(q)
    return lagrange_matrix(xp, xq)


def collapsed_triangle_rule(m: int):
    """(xi, eta, w) of the collapsed Gauss rule on the reference triangle
    {xi, eta >= 0, xi + eta <= 1}: xi = u, eta = (1 - u) v with u, v on m-point
    Gauss-Legendre rules of [0, 1] and weight (1 - u) w_u w_v. Exact for total
    degree 2m - 2; all weights positive; sum of weights 1/2."""
    t, wt = np.polynomial.legendre.leggauss(m)
    u = (t + 1) / 2
    wu = wt / 2
    U, Vv = np.meshgrid(u, u, indexing="ij")
    WU, WV = np.meshgrid(wu, wu, indexing="ij")
    xi = U.ravel()
    eta = ((1 - U) * Vv).ravel()
    w = ((1 - U) * WU * WV).ravel()
    return xi, eta, w


def triangle_upsample(p: int, xi_q, eta_q) -> np.ndarray:
    """O_{p,q} for triangles: values at the p-node set of setup.simplex (degree
    p - 1) to values of the same polynomial at (xi_q, eta_q): [n_q, p(p+1)/2]."""
    xi_p, eta_p, _ = simplex.simplex_rule(p)
    Vp = simplex.orthogonal_basis(xi_p, eta_p, p - 1)    # [n_p, n_p] values of the basis at the p-nodes
    Vq = simplex.orthogonal_basis(np.asarray(xi_q), np.asarray(eta_q), p - 1)
    return Vq @ np.linalg.inv(Vp)


@dataclass
class Upsampling:
    """Per-cell upsampling description (what the C ABI takes).

    types: list of dicts {"kind": "tensor", "a": [qa, pa], "b": [qb, pb]} (O = a kron b)
           or {"kind": "dense", "mat": [n_q, n_p]}
    cell_type [n_cells] int32, f_start [n_cells + 1] int64 (p-node ranges in the
    density), src_start [n_cells + 1] int64 (q-node ranges in the FMM sources).
    """

    types: list
    cell_type: np.ndarray
    f_start: np.ndarray
    src_start: np.ndarray

    @property
    def n_f(self) -> int:
        return int(self.f_start[-1])

    @property
    def n_q(self) -> int:
        return int(self.src_start[-1])

    def dense(self, t: int) -> np.ndarray:
        ty = self.types[t]
        return np.kron(ty["a"], ty["b"]) if ty["kind"] == "tensor" else ty["mat"]


def box_grid_upsampled(nbox: int, p: int = 8, q: int = 16, lo: float = -1.0, hi: float = 1.0):
    """q-nodes and weights of an nbox x nbox box grid (cell by cell, y-major,
    x fastest, like inputs.box_grid_nodes) and the Upsampling from the p x p
    nodes. Returns (xy_q [nbox^2 q^2, 2], w_q, Upsampling)."""
    tq, wq = np.polynomial.legendre.leggauss(q)
    side = (hi - lo) / nbox
    half = side / 2.0
    c = lo + half + side * np.arange(nbox)
    by, bx, iy, ix = np.meshgrid(np.arange(nbox), np.arange(nbox), np.arange(q), np.arange(q), indexing="ij")
    xy = np.stack([(c[bx] + half * tq[ix]).ravel(), (c[by] + half * tq[iy]).ravel()], axis=1)
    w = (wq[ix] * wq[iy] * half * half).ravel()
    L = box_upsample_1d(p, q)
    ncell = nbox * nbox
    ups = Upsampling(types=[{"kind": "tensor", "a": L, "b": L}], cell_type=np.zeros(ncell, np.int32),
                     f_start=np.arange(ncell + 1, dtype=np.int64) * p * p,
                     src_start=np.arange(ncell + 1, dtype=np.int64) * q * q)
    return np.ascontiguousarray(xy), w, ups


def apply(ups: Upsampling, f: np.ndarray) -> np.ndarray:
    """f_q = O f per cell, for f [ndens, n_f] (plain per-cell products)."""
    f = np.atleast_2d(f)
    out = np.empty((f.shape[0], ups.n_q))
    mats = [ups.dense(t) for t in range(len(ups.types))]
    for k in range(ups.cell_type.size):
        O = mats[ups.cell_type[k]]
        out[:, ups.src_start[k]:ups.src_start[k + 1]] = f[:, ups.f_start[k]:ups.f_start[k + 1]] @ O.T
    return out


def mesh_upsampling(mesh_p, mesh_q, p_box: int, q_box: int, p_tri: int, tri_q_rule) -> Upsampling:
    """Upsampling between two meshes of the same cells (same order and kinds):
    mesh_p with p_box^2 GL box nodes and p_tri-node simplex triangles, mesh_q with
    q_box^2 GL box nodes and the given triangle rule."""
    if not np.array_equal(mesh_p.cell_kind, mesh_q.cell_kind):
        raise ValueError("meshes have different cells")
    L = box_upsample_1d(p_box, q_box)
    types = [{"kind": "tensor", "a": L, "b": L},
             {"kind": "dense", "mat": triangle_upsample(p_tri, tri_q_rule[0], tri_q_rule[1])}]
    cell_type = np.where(mesh_p.cell_kind == 0, 0, 1).astype(np.int32)
    return Upsampling(types=types, cell_type=cell_type, f_start=np.asarray(mesh_p.cell_start, np.int64),
                      src_start=np.asarray(mesh_q.cell_start, np.int64))


__all__ = ["lagrange_matrix", "box_upsample_1d", "collapsed_triangle_rule", "triangle_upsample", "Upsampling",
           "box_grid_upsampled", "apply", "mesh_upsampling"]
