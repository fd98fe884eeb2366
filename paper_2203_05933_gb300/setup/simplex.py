"""Interpolation/quadrature nodes on the reference simplex and the triangle maps.

Reference simplex T0 = {(xi, eta): xi, eta >= 0, xi + eta <= 1} (Sec. 3.2.1).

The paper uses Vioreanu-Rokhlin nodes (Sec. 3.2.1, Eq. vio_rokh_quad_rule);
their tables are not available here, so this module builds its own stand-in
with the same roles: p(p+1)/2 interior nodes that are unisolvent for total
degree p-1 (approximate Fekete points, chosen greedily by column-pivoted QR of
an orthogonal-basis Vandermonde over a fine interior candidate lattice, in the
manner of Sommariva and Vianello), and interpolatory weights that integrate
every polynomial of total degree p-1 exactly (moment matching).

Maps (Sec. 3.2.1): the affine map of a straight triangle, and the blending map
of a curved triangle whose edge between vertices 1 and 2 follows a parametric
curve (lambda(xi), mu(xi)) (Eq. deformed_triangle_maps), with its Jacobian.
"""

from __future__ import annotations

import functools
import math

import numpy as np
import scipy.linalg
from scipy.special import eval_jacobi, eval_legendre


def orthogonal_basis(xi, eta, degree: int) -> np.ndarray:
    """Collapsed-coordinate orthogonal (Dubiner/Koornwinder-type) basis on T0,
    all total degrees <= degree. Returns V [npts, nbasis], evaluated without
    division: P_m(a) (1 - eta)^m is expanded as a polynomial in (xi, eta)."""
    xi = np.asarray(xi, float)
    eta = np.asarray(eta, float)
    b = 2.0 * eta - 1.0
    cols = []
    one_m_eta = 1.0 - eta
    for m in range(degree + 1):
        # P_m(a) (1-eta)^m with a (1-eta) = 2 xi - 1 + eta
        coef = np.polynomial.legendre.leg2poly(np.eye(m + 1)[m])
        s = 2.0 * xi - 1.0 + eta
        pm = sum(coef[i] * s**i * one_m_eta ** (m - i) for i in range(m + 1))
        for k in range(degree - m + 1):
            cols.append(pm * eval_jacobi(k, 2 * m + 1, 0, b))
    return np.stack(cols, axis=1)


def simplex_moments(degree: int) -> np.ndarray:
    """Integrals over T0 of the basis above, by a collapsed Gauss product rule
    exact for these polynomials."""
    n = degree + 2
    t, wt = np.polynomial.legendre.leggauss(n)
    u = 0.5 * (t + 1.0)
    wu = 0.5 * wt
    # Duffy: xi = u (1 - v), eta = v, Jacobian (1 - v)
    U, Vv = np.meshgrid(u, u, indexing="ij")
    W = np.outer(wu, wu) * (1.0 - Vv)
    xi = (U * (1.0 - Vv)).ravel()
    eta = Vv.ravel()
    return orthogonal_basis(xi, eta, degree).T @ W.ravel()


@functools.lru_cache(maxsize=None)
def simplex_rule(p: int, tries: int = 200, margin: float = 0.03):
    """(xi, eta, w) of p(p+1)/2 interior nodes unisolvent for degree p-1, with
    weights exact for all polynomials of total degree p-1 (sum w = 1/2).

    Greedy approximate-Fekete selection (column-pivoted QR of the transposed
    Vandermonde) over seeded random interior candidate sets; among the
    selections whose interpolatory weights are all positive, the one with the
    best-conditioned Vandermonde is kept. Deterministic."""
    degree = p - 1
    n = p * (p + 1) // 2
    moments = simplex_moments(degree)
    best = None
    for seed in range(tries):
        rng = np.random.default_rng(seed)
        u = rng.random((max(4000, 60 * n), 2))
        u = u[u.sum(axis=1) < 1.0]
        xi = margin + (1.0 - 3.0 * margin) * u[:, 0]
        eta = margin + (1.0 - 3.0 * margin) * u[:, 1]
        V = orthogonal_basis(xi, eta, degree)
        _, _, piv = scipy.linalg.qr(V.T, pivoting=True, mode="economic")
        sel = np.sort(piv[:n])
        Vn = orthogonal_basis(xi[sel], eta[sel], degree)
        w = np.linalg.solve(Vn.T, moments)
        if w.min() <= 0.0:
            continue
        cond = np.linalg.cond(Vn)
        if best is None or cond < best[0]:
            best = (cond, xi[sel].copy(), eta[sel].copy(), w)
    if best is None:
        raise RuntimeError(f"no positive-weight node set found for p={p}")
    return best[1], best[2], best[3]


def affine_map(v, xi, eta):
    """Straight triangle with vertices v [3, 2]: points [n, 2] and constant Jacobian."""
    v = np.asarray(v, float)
    x = (1 - xi - eta)[:, None] * v[0] + xi[:, None] * v[1] + eta[:, None] * v[2]
    J = abs((v[1, 0] - v[0, 0]) * (v[2, 1] - v[0, 1]) - (v[2, 0] - v[0, 0]) * (v[1, 1] - v[0, 1]))
    return x, np.full(xi.shape, J)


def blended_map_jacobian(v, curve, xi, eta):
    """The blending map of a curved triangle (as blended_map) and its partial
    derivatives: returns (x, y, x_xi, y_xi, x_eta, y_eta)."""
    v = np.asarray(v, float)
    lam, mu, dlam, dmu = curve(xi)
    g = (1 - xi - eta) / (1 - xi)
    phx = lam - (1 - xi) * v[0, 0] - xi * v[1, 0]
    phy = mu - (1 - xi) * v[0, 1] - xi * v[1, 1]
    x = (1 - xi - eta) * v[0, 0] + xi * v[1, 0] + eta * v[2, 0] + g * phx
    y = (1 - xi - eta) * v[0, 1] + xi * v[1, 1] + eta * v[2, 1] + g * phy
    dg_dxi = -eta / (1 - xi) ** 2
    x_xi = v[1, 0] - v[0, 0] + dg_dxi * phx + g * (dlam + v[0, 0] - v[1, 0])
    y_xi = v[1, 1] - v[0, 1] + dg_dxi * phy + g * (dmu + v[0, 1] - v[1, 1])
    x_eta = v[2, 0] - v[0, 0] - phx / (1 - xi)
    y_eta = v[2, 1] - v[0, 1] - phy / (1 - xi)
    return x, y, x_xi, y_xi, x_eta, y_eta


def blended_map(v, curve, xi, eta, signed: bool = False):
    """Curved triangle (Eq. deformed_triangle_maps): vertices v [3, 2], the edge
    from v[0] to v[1] follows curve(s) -> (lam, mu, dlam, dmu) for s in [0, 1]
    with curve(0) = v[0], curve(1) = v[1]. Returns points [n, 2] and |det DR|
    (det DR itself with signed=True)."""
    v = np.asarray(v, float)
    lam, mu, dlam, dmu = curve(xi)
    g = (1 - xi - eta) / (1 - xi)
    phx = lam - (1 - xi) * v[0, 0] - xi * v[1, 0]
    phy = mu - (1 - xi) * v[0, 1] - xi * v[1, 1]
    x = (1 - xi - eta) * v[0, 0] + xi * v[1, 0] + eta * v[2, 0] + g * phx
    y = (1 - xi - eta) * v[0, 1] + xi * v[1, 1] + eta * v[2, 1] + g * phy
    dg_dxi = -eta / (1 - xi) ** 2
    x_xi = v[1, 0] - v[0, 0] + dg_dxi * phx + g * (dlam + v[0, 0] - v[1, 0])
    y_xi = v[1, 1] - v[0, 1] + dg_dxi * phy + g * (dmu + v[0, 1] - v[1, 1])
    x_eta = v[2, 0] - v[0, 0] - phx / (1 - xi)
    y_eta = v[2, 1] - v[0, 1] - phy / (1 - xi)
    J = x_xi * y_eta - x_eta * y_xi
    return np.stack([x, y], axis=1), (J if signed else np.abs(J))


def circle_arc(cx, cy, r, th0, th1):
    """Arc of the circle (cx, cy, r) from angle th0 to th1, as a curve on [0, 1]."""
    dth = th1 - th0

    def curve(s):
        th = th0 + s * dth
        return (cx + r * np.cos(th), cy + r * np.sin(th), -r * dth * np.sin(th), r * dth * np.cos(th))

    curve.spec = (1.0, cx, cy, r, th0, th1)
    return curve


def gauss_legendre_box(order: int):
    t, w = np.polynomial.legendre.leggauss(order)
    X, Y = np.meshgrid(t, t, indexing="xy")
    WW = np.outer(w, w)
    return X.ravel(), Y.ravel(), WW.ravel()


def triangle_count_nodes(p: int) -> int:
    return p * (p + 1) // 2


__all__ = ["orthogonal_basis", "simplex_moments", "simplex_rule", "affine_map", "blended_map",
           "circle_arc", "gauss_legendre_box", "triangle_count_nodes", "math"]
