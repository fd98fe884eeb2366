"""Host set-up of the singular and near-singular corrections for box cells by
the area-to-line conversion of the paper (untimed; produces the correction
matrix that the hot path applies).

For a box B = c + a [-1, 1]^2 and a target t = c + a z0 (z0 in reference
coordinates), the accurate potential of a basis function rho on B is

    a^2 int_{B0} G(a (z - z0)) rho(z) dz,    G(r) = -(1/2pi) log|r|   (Sec. 2.1),

turned into line integrals over the boundary of B0 (Lemma 1 and its corollary,
Sec. 3.3; Eq. Vk_bdry_quad): with a star point z* (z* = z0 for targets inside
the box, else the point of B0 closest to z0, Eq. rstar_def),

    int_{B0} K(z - z0) rho(z) dz
        = sum_edges  D_e int_0^1 I(z_b(s)) ds,
    I(z_b) = int_0^1 t K(z* + t (z_b - z*) - z0) rho(z* + t (z_b - z*)) dt,

where z_b(s) runs along the edge from P0 to P1 and D_e = (P0 - z*) x (P1 - P0)
is constant on the edge (edges through z* drop out). For self targets the
inner integrand is t (log t + log|z_b - z0|) rho: the log t part is integrated
by a Gauss rule for the weight -log t (the role of the paper's endpoint-
corrected rules, Eq. Ik_vp_singular), the rest by Gauss-Legendre; for near
targets the inner integrand is smooth but steep at t = 0 and is integrated by
Gauss-Legendre on panels graded towards t = 0 (the role of the paper's
near-singular rules, Eq. near_sing_dist_rule). The outer s integrals use
Gauss-Legendre on panels graded towards the point of the edge nearest to z0
(the target-adapted panels of Sec. 3.3.3).

Basis: tensor Legendre polynomials P_m(x) P_n(y), m, n < order, mapped to the
nodal (Lagrange) basis of the order x order Gauss-Legendre nodes by the inverse
Vandermonde matrix (the coefficient map of Eq. amap_koorn / Eq.
mapbox_singular_quad with a Legendre in place of a Chebyshev basis). The
correction of node j for target t is "accurate minus smooth" (Sec. 4): the
basis potential minus the smooth-rule term a^2 w_j G(r_j - t), the latter
omitted when r_j = t.

By translation invariance (Eq. Vkhat_box) the corrections of a uniform grid are
one lookup table per neighbour offset (Sec. 4.2), with the box size entering
only through a log(a) term.
"""

from __future__ import annotations

import functools
import math

import numpy as np

INV_2PI = 1.0 / (2.0 * math.pi)


@functools.lru_cache(maxsize=None)
def log_weight_rule(n: int):
    """Gauss rule for int_0^1 -log(t) g(t) dt, exact for polynomials of degree
    2n - 1 (Golub-Welsch from the moments 1/(k+1)^2, Cholesky of the Hankel
    moment matrix in 100-digit arithmetic)."""
    import mpmath

    with mpmath.workdps(100):
        N = n + 1
        H = mpmath.matrix(N, N)
        for i in range(N):
            for j in range(N):
                H[i, j] = mpmath.mpf(1) / (i + j + 1) ** 2
        R = mpmath.cholesky(H).T  # upper triangular, H = R^T R
        alpha = []
        beta = []
        for k in range(n):
            a = R[k, k + 1] / R[k, k] - (R[k - 1, k] / R[k - 1, k - 1] if k > 0 else 0)
            alpha.append(a)
            if k < n - 1:
                beta.append(R[k + 1, k + 1] / R[k, k])
        J = np.diag([float(a) for a in alpha]) + np.diag([float(b) for b in beta], 1) + \
            np.diag([float(b) for b in beta], -1)
        evals, evecs = np.linalg.eigh(J)
        w = evecs[0, :] ** 2 * 1.0  # mu_0 = int -log t dt = 1
    return evals, w


@functools.lru_cache(maxsize=None)
def gl01(n: int):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def graded_panels(p: float, scale: float, lo: float = 0.0, hi: float = 1.0, ratio: float = 0.25,
                  nlev: int = 40):
    """Panel breakpoints of [lo, hi] graded geometrically (ratio) towards p,
    down to panels of about `scale`."""
    p = min(max(p, lo), hi)
    pts = {lo, hi, p}
    for side in (-1.0, 1.0):
        end = lo if side < 0 else hi
        span = abs(end - p)
        width = span
        x = p
        level = 0
        while width > max(scale, 1e-14) and level < nlev:
            width *= ratio
            pts.add(p + side * width)
            level += 1
    return np.array(sorted(x for x in pts if lo <= x <= hi))


def composite_rule(breaks, n: int = 16):
    t, w = gl01(n)
    h = np.diff(breaks)
    x = (breaks[:-1, None] + h[:, None] * t[None, :]).ravel()
    ww = (h[:, None] * w[None, :]).ravel()
    return x, ww


def legendre_basis(x, y, order: int):
    """[npts, order*order] values of P_m(x) P_n(y), column m*order + n."""
    V = np.polynomial.legendre.legvander2d(np.asarray(x, float), np.asarray(y, float), [order - 1, order - 1])
    return V


@functools.lru_cache(maxsize=None)
def gl_box(order: int):
    """order x order Gauss-Legendre nodes of [-1,1]^2 (x fastest, as in the box
    grid generator), weights, and the nodal map C (Legendre coefficients ->
    values inverted): nodal potential = legendre potentials @ C."""
    t, w = np.polynomial.legendre.leggauss(order)
    X, Y = np.meshgrid(t, t, indexing="xy")
    x, y = X.ravel(), Y.ravel()
    W = np.outer(w, w).ravel()
    V = legendre_basis(x, y, order)  # V[i, mn] = phi_mn(node i)
    return x, y, W, np.linalg.inv(V)


_EDGES = (((-1.0, -1.0), (1.0, -1.0)), ((1.0, -1.0), (1.0, 1.0)), ((1.0, 1.0), (-1.0, 1.0)),
          ((-1.0, 1.0), (-1.0, -1.0)))


def box_basis_potentials(z0, order: int = 8, n_t: int = 16, n_s: int = 16) -> np.ndarray:
    """int_{[-1,1]^2} G(z - z0) P_m(x) P_n(y) dz for all m, n < order
    (G = -(1/2pi) log|.|, unit scale), by the area-to-line conversion."""
    z0 = np.asarray(z0, float)
    inside = abs(z0[0]) <= 1.0 and abs(z0[1]) <= 1.0
    zs = z0.copy() if inside else np.clip(z0, -1.0, 1.0)
    dist = 0.0 if inside else float(np.hypot(*(z0 - zs)))
    total = np.zeros(order * order)
    if inside:
        tl, wl = log_weight_rule(n_t)
        tg, wg = gl01(n_t)
    for P0, P1 in _EDGES:
        P0 = np.array(P0)
        P1 = np.array(P1)
        e = P1 - P0
        D = (P0[0] - zs[0]) * e[1] - (P0[1] - zs[1]) * e[0]
        if abs(D) < 1e-15:
            continue
        # foot of z0 on the edge line and its distance
        L2 = float(e @ e)
        sf = float((z0 - P0) @ e) / L2
        foot = P0 + min(max(sf, 0.0), 1.0) * e
        dline = float(np.hypot(*(z0 - foot)))
        s, ws = composite_rule(graded_panels(sf, max(dline, 1e-3) / math.sqrt(L2) * 0.5), n_s)
        zb = P0[None, :] + s[:, None] * e[None, :]
        v = zb - zs[None, :]
        vn = np.hypot(v[:, 0], v[:, 1])
        if inside:
            # int_0^1 t (log t + log|v|) rho(z0 + t v) dt
            pl = zs[None, None, :] + tl[None, :, None] * v[:, None, :]
            pg = zs[None, None, :] + tg[None, :, None] * v[:, None, :]
            Bl = legendre_basis(pl[..., 0].ravel(), pl[..., 1].ravel(), order).reshape(len(s), n_t, -1)
            Bg = legendre_basis(pg[..., 0].ravel(), pg[..., 1].ravel(), order).reshape(len(s), n_t, -1)
            Ilog = -np.einsum("m,m,smk->sk", wl, tl, Bl)  # int t log t rho dt
            Ismooth = np.einsum("m,m,smk->sk", wg, tg, Bg)
            I = -INV_2PI * (Ilog + np.log(vn)[:, None] * Ismooth)
        else:
            # smooth but steep at t = 0: panels graded towards 0 with scale dist / |v|
            I = np.zeros((len(s), order * order))
            for k in range(len(s)):
                tb, wb = composite_rule(graded_panels(0.0, dist / max(vn[k], 1e-300) * 0.5), n_t)
                pts = zs[None, :] + tb[:, None] * v[k][None, :]
                r = np.hypot(pts[:, 0] - z0[0], pts[:, 1] - z0[1])
                B = legendre_basis(pts[:, 0], pts[:, 1], order)
                I[k] = (wb * tb * (-INV_2PI) * np.log(r)) @ B
        total += D * (ws @ I)
    return total


def box_node_corrections(z0, a: float = 1.0, order: int = 8, coincident: int | None = None,
                         q: int | None = None) -> np.ndarray:
    """Correction weights (accurate minus smooth) of the order^2 GL nodes of the
    box c + a[-1,1]^2 for the target c + a z0. `coincident` is the index of the
    node equal to the target, if any (its smooth term is omitted).
    q: the smooth rule is the oversampled one (Sec. 2, "Oversampled smooth
    quadratures"; Sec. 4.2): q x q GL nodes carrying the values interpolated
    from the order x order nodes, so the smooth weight of node i is
    sum_j W^q_j G(z^q_j, z0) O_ji. The q-nodes never coincide with a p-node
    target (disjoint Gauss-Legendre sets)."""
    x, y, W, Vinv = gl_box(order)
    pot = box_basis_potentials(z0, order) @ Vinv  # nodal potentials at unit scale
    if q is not None:
        from .upsample import box_upsample_1d

        xq, yq, Wq, _ = gl_box(q)
        L = box_upsample_1d(order, q)
        rq = np.hypot(xq - z0[0], yq - z0[1])
        if np.any(rq == 0.0):
            raise ValueError("target on an oversampled node")
        smooth = (Wq * (-INV_2PI) * np.log(rq)) @ np.kron(L, L)
        return a * a * (pot - smooth)  # log a terms cancel: both rules integrate the nodal basis exactly
    r = np.hypot(x - z0[0], y - z0[1])
    corr = np.empty(order * order)
    with np.errstate(divide="ignore"):
        smooth_unit = W * (-INV_2PI) * np.log(r)
    corr[:] = pot - smooth_unit  # the log a terms of accurate and smooth cancel
    if coincident is not None:
        corr[coincident] = pot[coincident] - INV_2PI * math.log(a) * W[coincident]
    return a * a * corr


def box_grid_correction_tables(order: int = 8, a: float = 1.0, q: int | None = None) -> np.ndarray:
    """T[oy+1, ox+1, i, j]: correction of source node j of a box for target
    node i of the box at offset (ox, oy) in {-1, 0, 1}^2 (uniform grid, half
    side a). One table per offset serves every box (Eq. Vkhat_box).
    q: oversampled smooth rule (see box_node_corrections)."""
    x, y, W, _ = gl_box(order)
    n = order * order
    T = np.empty((3, 3, n, n))
    for oy in (-1, 0, 1):
        for ox in (-1, 0, 1):
            for i in range(n):
                z0 = np.array([x[i] + 2.0 * ox, y[i] + 2.0 * oy])
                T[oy + 1, ox + 1, i] = box_node_corrections(z0, a, order,
                                                            coincident=i if (ox == 0 and oy == 0) else None, q=q)
    return T


def box_grid_csr(nbox: int, order: int = 8, lo: float = -1.0, hi: float = 1.0, tables=None, q: int | None = None):
    """Correction matrix of the nbox x nbox box grid on [lo, hi]^2 with order^2
    GL nodes per box, in the node order of the box-grid generator (cell by
    cell, x fastest) and the own + 8 neighbour pattern. Rows are the p-node
    targets, columns the p-nodes (the density samples), also with an
    oversampled smooth rule (q)."""
    a = (hi - lo) / nbox / 2.0
    T = box_grid_correction_tables(order, a, q) if tables is None else tables
    npc = order * order
    rows_ptr = [0]
    cols, vals = [], []
    for by in range(nbox):
        for bx in range(nbox):
            nb = [(ny, nx) for ny in range(max(0, by - 1), min(nbox, by + 2))
                  for nx in range(max(0, bx - 1), min(nbox, bx + 2))]
            for i in range(npc):
                for ny, nx in nb:
                    c = ny * nbox + nx
                    cols.append(np.arange(c * npc, (c + 1) * npc, dtype=np.int32))
                    # target box is at offset (bx - nx, by - ny) from the source box
                    vals.append(T[by - ny + 1, bx - nx + 1, i])
                rows_ptr.append(rows_ptr[-1] + npc * len(nb))
    return np.array(rows_ptr, np.int64), np.concatenate(cols), np.concatenate(vals)


def box_grid_corrections_at(targets, nbox: int, order: int = 8, lo: float = -1.0, hi: float = 1.0):
    """Correction rows for arbitrary targets inside the box grid (the generic,
    target-dependent pre-computation of Sec. 4): each target couples to the
    nodes of the box containing it and of the (up to) 8 boxes around it.
    Returns CSR (rowptr, col, val) with columns in the grid's node order."""
    targets = np.asarray(targets, float).reshape(-1, 2)
    side = (hi - lo) / nbox
    a = side / 2.0
    x, y, _, _ = gl_box(order)
    npc = order * order
    lens, cols, vals = [], [], []
    for t in targets:
        bx = min(max(int((t[0] - lo) // side), 0), nbox - 1)
        by = min(max(int((t[1] - lo) // side), 0), nbox - 1)
        n_blocks = 0
        for ny in range(max(0, by - 1), min(nbox, by + 2)):
            for nx in range(max(0, bx - 1), min(nbox, bx + 2)):
                c = ny * nbox + nx
                cx, cy = lo + (nx + 0.5) * side, lo + (ny + 0.5) * side
                z0 = np.array([(t[0] - cx) / a, (t[1] - cy) / a])
                coinc = np.nonzero((cx + a * x == t[0]) & (cy + a * y == t[1]))[0]
                cols.append(np.arange(c * npc, (c + 1) * npc, dtype=np.int32))
                vals.append(box_node_corrections(z0, a, order, coincident=int(coinc[0]) if coinc.size else None))
                n_blocks += 1
        lens.append(n_blocks * npc)
    rp = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    return rp, np.concatenate(cols), np.concatenate(vals)
