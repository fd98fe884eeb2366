"""Triangle self-correction rules (host set-up): the fixed reference-space rule
of each target node reproduces the basis potentials of curved and straight
cells. Curved: scipy's adaptive 2-D quadrature over the three sub-triangles
that meet at the target (scalar integrand). Straight (affine map): the inner
ray integral in closed form, int_0^1 t log(t |A v|) dt = -1/4 + log|A v| / 2,
and the edge integral by mpmath. The rule is the same for every cell, so its
panels follow reference-space distances: its accuracy presumes well-shaped
cells (about 1e-13 at a smallest angle of 30 degrees, 1e-11 at 20, 1e-7 at
8 on straight cells), as the paper's meshes provide."""

import math

import mpmath
import numpy as np
import scipy.integrate as si
from scipy.special import eval_jacobi, eval_legendre

from paper_2203_05933_gb300.setup import meshes, simplex, tricorr


def _scalar_blended(v, spec):
    """Scalar blending map of a circle-arc triangle: (xi, eta) -> (x, y, J)."""
    _, cx, cy, r, th0, th1 = spec
    dth = th1 - th0

    def f(xi, eta):
        th = th0 + xi * dth
        lam, mu = cx + r * math.cos(th), cy + r * math.sin(th)
        dl, dm = -r * dth * math.sin(th), r * dth * math.cos(th)
        om = 1.0 - xi
        g = (1.0 - xi - eta) / om
        phx = lam - om * v[0][0] - xi * v[1][0]
        phy = mu - om * v[0][1] - xi * v[1][1]
        x = (1 - xi - eta) * v[0][0] + xi * v[1][0] + eta * v[2][0] + g * phx
        y = (1 - xi - eta) * v[0][1] + xi * v[1][1] + eta * v[2][1] + g * phy
        dg = -eta / om ** 2
        x_xi = v[1][0] - v[0][0] + dg * phx + g * (dl + v[0][0] - v[1][0])
        y_xi = v[1][1] - v[0][1] + dg * phy + g * (dm + v[0][1] - v[1][1])
        x_eta = v[2][0] - v[0][0] - phx / om
        y_eta = v[2][1] - v[0][1] - phy / om
        return x, y, abs(x_xi * y_eta - x_eta * y_xi)

    return f


def _K(xi, eta, m, k):
    s, t = 2 * xi - 1 + eta, 1 - eta
    return eval_legendre(m, s / t) * t ** m * eval_jacobi(k, 2 * m + 1, 0, 2 * eta - 1)


def _vhat(R, fmap_vec, a):
    z0 = (R["xi"][a], R["eta"][a])
    x0, y0, _ = fmap_vec(z0[0], z0[1])
    x, y, J = fmap_vec(R["chi"][a][:, 0], R["chi"][a][:, 1])
    return R["B"][a] @ tricorr.kernel_factor(x, y, J, x0[0], y0[0], R["tau"][a])


def test_self_rule_matches_adaptive_quadrature_on_a_curved_cell():
    m = meshes.disk_mesh(base_level=3, fine_level=3)
    k = [i for i, g in enumerate(m.geom) if g[0] == "tri" and g[2] is not None][2]
    _, v, curve = m.geom[k]
    R = tricorr.self_rules(8)
    a, (mm, kk), b = 4, (2, 1), None
    # basis column of (m, k) = (2, 1): columns run over m, then k = 0..7-m
    b = sum(8 - q for q in range(mm)) + kk
    vh = _vhat(R, tricorr.cell_map(m.geom[k]), a)[b]
    f = _scalar_blended(v, curve.spec)
    z0 = np.array([R["xi"][a], R["eta"][a]])
    x0, y0, _ = f(*z0)
    P = [np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.0, 1.0])]
    tot = 0.0
    for e in range(3):
        A, B = P[e], P[(e + 1) % 3]
        cr = abs((A[0] - z0[0]) * (B[1] - A[1]) - (A[1] - z0[1]) * (B[0] - A[0]))

        def F(vv, u, A=A, B=B, cr=cr):
            xi, eta = z0 + u * (A + vv * (B - A) - z0)
            x, y, J = f(xi, eta)
            return u * cr * (-math.log(math.hypot(x - x0, y - y0)) / (2 * math.pi)) * J * _K(xi, eta, mm, kk)

        tot += si.dblquad(F, 0, 1, 0, 1, epsabs=1e-16, epsrel=1e-12)[0]
    assert abs(vh - tot) <= 1e-12 * max(1e-3, abs(tot)), (vh, tot)


def _min_angle(v):
    out = []
    for i in range(3):
        u, w = v[(i + 1) % 3] - v[i], v[(i + 2) % 3] - v[i]
        out.append(math.degrees(math.acos(np.clip(u @ w / np.linalg.norm(u) / np.linalg.norm(w), -1, 1))))
    return min(out)


def test_self_rule_on_a_straight_cell_against_the_reduced_integral():
    m = meshes.disk_mesh(base_level=3, fine_level=3)
    k = [i for i, g in enumerate(m.geom) if g[0] == "tri" and g[2] is None and _min_angle(g[1]) >= 30.0][0]
    _, v, _ = m.geom[k]
    R = tricorr.self_rules(8)
    A = np.array([[v[1, 0] - v[0, 0], v[2, 0] - v[0, 0]], [v[1, 1] - v[0, 1], v[2, 1] - v[0, 1]]])
    Jc = abs(np.linalg.det(A))
    c0 = simplex.orthogonal_basis(np.array([0.3]), np.array([0.3]), 7)[0, 0]  # K_0 is constant
    P = [np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.0, 1.0])]
    for a in (4, 22, 30):
        z0 = np.array([R["xi"][a], R["eta"][a]])
        tot = mpmath.mpf(0)
        for e in range(3):
            Pa, Pb = P[e], P[(e + 1) % 3]
            D = (Pa[0] - z0[0]) * (Pb[1] - Pa[1]) - (Pa[1] - z0[1]) * (Pb[0] - Pa[0])

            def inner(s, Pa=Pa, Pb=Pb):
                ph = A @ (Pa + float(s) * (Pb - Pa) - z0)
                return -mpmath.mpf(1) / 4 + mpmath.log(mpmath.hypot(ph[0], ph[1])) / 2

            tot += D * mpmath.quad(inner, [0, 1])
        exact = float(-tot / (2 * mpmath.pi)) * Jc * c0
        vh = _vhat(R, tricorr.cell_map(m.geom[k]), a)[0]
        assert abs(vh - exact) <= 1e-12 * abs(exact), (a, vh, exact)


def test_self_block_reproduces_constant_density_potential():
    # sum_j corr[a, j] + the smooth rule's terms = the accurate potential of
    # f = 1 over the cell at its node a, i.e. Vhat[K_0] / K_0
    m = meshes.disk_mesh(base_level=3, fine_level=3)
    k = [i for i, g in enumerate(m.geom) if g[0] == "tri" and g[2] is not None][5]
    R = tricorr.self_rules(8)
    corr = tricorr.self_corrections_reference(m.geom[k], R)
    fmap = tricorr.cell_map(m.geom[k])
    xn, yn, Jn = fmap(R["xi"], R["eta"])
    k0 = simplex.orthogonal_basis(np.array([0.3]), np.array([0.3]), 7)[0, 0]
    for a in (0, 11, 35):
        r = np.hypot(xn - xn[a], yn - yn[a])
        smooth = sum(R["tw"][j] * Jn[j] * (-math.log(r[j]) / (2 * math.pi)) for j in range(xn.size) if j != a)
        assert abs(corr[a].sum() + smooth - _vhat(R, fmap, a)[0] / k0) < 1e-14
