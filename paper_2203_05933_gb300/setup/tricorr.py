"""Reference-space rules for the singular (self) corrections of mapped
triangles (Sec. 3.3 and the efficient pre-computation of Sec. 3.4, Eq.
singcorr_inner_prod): for a target at a fixed reference node zeta_0 of the
simplex T0, the volume integral of G(R(zeta), R(zeta_0)) rho(zeta) J(zeta) over
T0 becomes, by the area-to-line conversion with star point zeta_0,

    sum_edges D_e int_0^1 ds int_0^1 t  G(R(zeta_0 + t v(s)), R(zeta_0)) rho J dt,
    v(s) = P_e(s) - zeta_0,  D_e = (P_e0 - zeta_0) x (P_e1 - P_e0),

and one fixed set of nodes chi_i and weights omega_i (the same for every cell)
discretises it:

    Vhat[K_b](zeta_0) ~ sum_i G(R(chi_i), R(zeta_0)) J(chi_i) K_b(chi_i) omega_i .

With the mapped distance written as t times a smooth factor, the Green
function splits into G = -(1/2pi) (log t + L(t)), L(t) = log(|R(zeta_0 + t v)
- R(zeta_0)| / t) smooth, so each ray carries two fixed t rules with positive
weights: the n-point Gauss rule for the weight -log t (for t log(t) J K) and
n-point Gauss-Legendre (for t L(t) J K). The cell-dependent factor at a node of
the first kind is J / (2 pi), at a node of the second kind -L J / (2 pi); in
both cases a mapped-Green-function-times-Jacobian value, and the rest,
B_b,i = K_b(chi_i) omega_i, is fixed. The s integrals use Gauss-Legendre on
panels graded towards the foot of zeta_0 on each edge.

Host set-up only; the evaluation runs in libvp (vp_tricorr_*).
"""

from __future__ import annotations

import functools
import math

import numpy as np

from . import simplex
from .corrections import composite_rule, graded_panels, log_weight_rule

INV_2PI = 1.0 / (2.0 * math.pi)


_EDGES_T0 = ((np.array([0.0, 0.0]), np.array([1.0, 0.0])), (np.array([1.0, 0.0]), np.array([0.0, 1.0])),
             (np.array([0.0, 1.0]), np.array([0.0, 0.0])))


def target_rule(z0, n_s: int = 16, n_t: int = 12):
    """Nodes chi [N, 2], signed ray parameters tau [N] and weights omega [N] of
    the self rule for target z0 inside T0 (star point z0). tau < 0 marks a
    node of the -log t rule (|tau| = t; its kernel factor is J / (2 pi)),
    tau > 0 a Gauss-Legendre node (kernel factor -L(t) J / (2 pi)); the t and
    polar-Jacobian factors are in omega."""
    z0 = np.asarray(z0, float)
    tl, wl = log_weight_rule(n_t)
    tg, wg = np.polynomial.legendre.leggauss(n_t)
    tg, wg = 0.5 * (tg + 1.0), 0.5 * wg
    tt = np.concatenate([np.asarray(tl), tg])
    wt = np.concatenate([np.asarray(wl) * np.asarray(tl), wg * tg])
    sign = np.concatenate([-np.ones(n_t), np.ones(n_t)])
    chis, taus, oms = [], [], []
    for P0, P1 in _EDGES_T0:
        e = P1 - P0
        D = (P0[0] - z0[0]) * e[1] - (P0[1] - z0[1]) * e[0]
        L2 = float(e @ e)
        sf = float((z0 - P0) @ e) / L2
        foot = P0 + min(max(sf, 0.0), 1.0) * e
        dline = float(np.hypot(*(z0 - foot)))
        s, ws = composite_rule(graded_panels(sf, max(dline, 1e-3) / math.sqrt(L2) * 0.5), n_s)
        pb = P0[None, :] + s[:, None] * e[None, :]
        v = pb - z0[None, :]
        chi = z0[None, None, :] + tt[None, :, None] * v[:, None, :]
        om = D * ws[:, None] * wt[None, :]
        chis.append(chi.reshape(-1, 2))
        taus.append(np.broadcast_to(sign * tt, (s.size, tt.size)).ravel())
        oms.append(om.ravel())
    return np.vstack(chis), np.concatenate(taus), np.concatenate(oms)


def kernel_factor(x, y, J, x0, y0, tau):
    """Cell-dependent factor of each node (see target_rule)."""
    t = np.abs(tau)
    L = np.log(np.hypot(x - x0, y - y0)) - np.log(t)
    return np.where(tau < 0, INV_2PI * J, -INV_2PI * L * J)


@functools.lru_cache(maxsize=None)
def self_rules(p: int = 8, n_s: int = 16, n_t: int = 12):
    """For every node a of the p-node simplex set: nodes chi_a, and
    B_a = K(chi_a)^T * omega_a ([n_basis, N_a]); plus the node set, reference
    weights and C = V^-1. All rules padded to the same length N (zero weights)."""
    xi, eta, tw = simplex.simplex_rule(p)
    Vn = simplex.orthogonal_basis(xi, eta, p - 1)
    C = np.linalg.inv(Vn)
    rules = [target_rule((xi[a], eta[a]), n_s, n_t) for a in range(xi.size)]
    N = max(r[0].shape[0] for r in rules)
    chi = np.zeros((xi.size, N, 2))
    tau = np.ones((xi.size, N))
    B = np.zeros((xi.size, Vn.shape[1], N))
    for a, (c, tu, om) in enumerate(rules):
        n = c.shape[0]
        chi[a, :n] = c
        tau[a, :n] = tu
        # padding: a node away from zeta_0 with weight zero
        chi[a, n:] = (xi[a], eta[a]) + np.array([0.1, 0.1]) * (1 - xi[a] - eta[a])
        B[a, :, :n] = (simplex.orthogonal_basis(c[:, 0], c[:, 1], p - 1) * om[:, None]).T
    return {"xi": xi, "eta": eta, "tw": tw, "C": C, "chi": chi, "tau": tau, "B": B, "N": N}


def cell_map(geom):
    """(map, curve-spec) for a triangle cell of setup.meshes: map(xi, eta) -> (x, y, J)."""
    _, v, curve = geom
    if curve is None:
        def f(xi, eta):
            pts, J = simplex.affine_map(v, np.atleast_1d(xi), np.atleast_1d(eta))
            return pts[:, 0], pts[:, 1], J
    else:
        def f(xi, eta):
            pts, J = simplex.blended_map(v, curve, np.atleast_1d(xi), np.atleast_1d(eta))
            return pts[:, 0], pts[:, 1], J
    return f


def self_corrections_reference(geom, rules) -> np.ndarray:
    """The self-correction block [n_nodes, n_nodes] of one triangle cell, by the
    rule (plain numpy): corr[a, j] = sum_b Vhat_a[b] C[b, j] minus the smooth
    rule's term w_j J(zeta_j) G(R(zeta_j), R(zeta_a)) (none for j = a)."""
    f = cell_map(geom)
    xi, eta, tw, C = rules["xi"], rules["eta"], rules["tw"], rules["C"]
    xn, yn, Jn = f(xi, eta)
    n = xi.size
    out = np.empty((n, n))
    for a in range(n):
        chi = rules["chi"][a]
        x, y, J = f(chi[:, 0], chi[:, 1])
        g = kernel_factor(x, y, J, xn[a], yn[a], rules["tau"][a])
        vhat = rules["B"][a] @ g
        r = np.hypot(xn - xn[a], yn - yn[a])
        with np.errstate(divide="ignore"):
            sm = tw * Jn * (-INV_2PI) * np.log(r)
        sm[a] = 0.0
        out[a] = vhat @ C - sm
    return out


def geom_params(geom, star_a: float = 0.3, star_k: int = 5):
    """12 doubles describing a triangle cell for the GPU: v0, v1, v2 (x, y),
    kind (0 straight, 1 circle arc, 2 star arc) and the curve parameters
    (circle: cx, cy, r, th0, th1; star: a, k, th0, th1). The curved edge runs
    from v0 to v1."""
    _, v, curve = geom
    out = np.zeros(12)
    out[:6] = np.asarray(v, float).ravel()
    if curve is None:
        return out
    spec = getattr(curve, "spec", None)
    if spec is None:
        raise ValueError("curved triangle without a curve description")
    out[6:6 + len(spec)] = spec
    return out
