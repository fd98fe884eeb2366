"""Host set-up (untimed): quadrature rules, meshes and the area-to-line box
corrections, pinned against facts independent of the code under test."""

import math

import numpy as np
import pytest
import scipy.integrate as si

import oracle
from paper_2203_05933_gb300 import inputs
from paper_2203_05933_gb300.setup import corrections as C
from paper_2203_05933_gb300.setup import meshes, simplex
from test_oracle_pins import rect_potential


def test_log_weight_rule_is_exact_to_degree_2n_minus_1():
    t, w = C.log_weight_rule(12)
    for k in range(24):  # int_0^1 -log(t) t^k dt = 1/(k+1)^2
        assert abs(np.sum(w * t**k) - 1.0 / (k + 1) ** 2) < 1e-15
    assert np.all(w > 0) and np.all((t > 0) & (t < 1))


def _brute_box_potential(z0, m, n):
    # scipy's adaptive 2-D quadrature on the square split at the target
    xs = [-1.0, 1.0] if not (-1 < z0[0] < 1) else [-1.0, z0[0], 1.0]
    ys = [-1.0, 1.0] if not (-1 < z0[1] < 1) else [-1.0, z0[1], 1.0]
    cm = np.zeros(m + 1)
    cm[m] = 1
    cn = np.zeros(n + 1)
    cn[n] = 1
    tot = 0.0
    for i in range(len(xs) - 1):
        for j in range(len(ys) - 1):
            v, _ = si.dblquad(lambda y, x: -math.log(math.hypot(x - z0[0], y - z0[1])) / (2 * math.pi)
                              * np.polynomial.legendre.legval(x, cm) * np.polynomial.legendre.legval(y, cn),
                              xs[i], xs[i + 1], ys[j], ys[j + 1], epsabs=1e-14, epsrel=1e-13)
            tot += v
    return tot


@pytest.mark.parametrize("z0", [(0.3, -0.2), (0.96028985649753623, 0.18343464249564981),
                                (1.0397101435024638, 0.52553240991632899), (1.2, 1.3)])
def test_area_to_line_basis_potentials_match_adaptive_quadrature(z0):
    z0 = np.array(z0)
    pot = C.box_basis_potentials(z0)
    for m, n in [(0, 0), (3, 5), (7, 7)]:
        assert abs(pot[m * 8 + n] - _brute_box_potential(z0, m, n)) < 1e-13


def test_corrected_box_grid_reproduces_constant_density_closed_form():
    # f = 1 on [-1,1]^2 (4x4 boxes, 8x8 GL): smooth rule + corrections at every node
    csr = C.box_grid_csr(4, 8)
    p = inputs.box_grid_problem(nbox=4, order=8, csr=csr)
    V = oracle.evaluate(p.src_xy, p.w, np.ones(p.n_src), p.tgt_xy, csr)
    ref = np.array([rect_potential(x, y, -1, 1, -1, 1) for x, y in p.tgt_xy])
    assert np.max(np.abs(V - ref)) < 1e-12
    V0 = oracle.evaluate(p.src_xy, p.w, np.ones(p.n_src), p.tgt_xy, None)
    assert np.max(np.abs(V0 - ref)) > 1e-3  # the corrections are what makes it exact


def test_corrected_box_grid_is_exact_for_polynomial_densities():
    # a degree-7 polynomial lies in every box's basis, so corrected values are exact
    def poly(x, y):
        return 1.0 + x**3 * y**2 - 2.0 * x * y**5 + 0.5 * x**7
    csr = C.box_grid_csr(2, 8)
    p = inputs.box_grid_problem(nbox=2, order=8, csr=csr)
    f = poly(p.src_xy[:, 0], p.src_xy[:, 1])
    idx = [0, 37, 100, 201]
    V = oracle.evaluate(p.src_xy, p.w, f, p.tgt_xy[idx], oracle.csr_rows(csr, idx))
    for k, i in enumerate(idx):
        x0, y0 = p.tgt_xy[i]
        tot = 0.0
        for xa, xb in ((-1.0, x0), (x0, 1.0)):
            for ya, yb in ((-1.0, y0), (y0, 1.0)):
                v, _ = si.dblquad(lambda y, x: -math.log(math.hypot(x - x0, y - y0)) / (2 * math.pi) * poly(x, y),
                                  xa, xb, ya, yb, epsabs=1e-14, epsrel=1e-13)
                tot += v
        assert abs(V[k] - tot) < 1e-12


def test_poisson_invariant_with_manufactured_source():
    # -Lap V = f inside the domain (V is the Newton potential of f), with f the
    # manufactured source of the paper's numerical results; corrections at
    # arbitrary (off-node) targets, 4th-order finite differences with h = 0.02
    def fman(x, y):
        return (6 * np.sin(6 * x) + 8 * np.cos(8 * (y + 0.1)) + 4 * (x * x + y * y) * np.sin(4 * x * y)
                + 3 * np.cos(3 * x) * np.sin(3 * y))
    nbox = 16
    xy, w, _ = inputs.box_grid_nodes(nbox, 8)
    f = fman(xy[:, 0], xy[:, 1])
    h = 0.02
    coef = np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / 12.0
    for pnt in ([0.13, -0.27], [-0.41, 0.38]):
        pnt = np.array(pnt)
        tg = np.array([pnt + [k * h, 0] for k in (-2, -1, 0, 1, 2)] + [pnt + [0, k * h] for k in (-2, -1, 0, 1, 2)])
        V = oracle.evaluate(xy, w, f, tg, C.box_grid_corrections_at(tg, nbox))
        lap = (coef @ V[:5] + coef @ V[5:]) / h**2
        assert abs(-lap - fman(*pnt)) < 2e-4
        V0 = oracle.evaluate(xy, w, f, tg, None)
        assert abs(-(coef @ V0[:5] + coef @ V0[5:]) / h**2 - fman(*pnt)) > 1e-2


def test_simplex_rule_is_interpolatory_of_degree_7_with_positive_weights():
    xi, eta, w = simplex.simplex_rule(8)
    assert xi.size == 36 and np.all(w > 0)
    for a in range(8):
        for b in range(8 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * xi**a * eta**b) - exact) < 1e-15
    V = simplex.orthogonal_basis(xi, eta, 7)
    assert np.linalg.cond(V) < 100  # unisolvent, well conditioned


def test_curved_triangle_map_area():
    xi, eta, w = simplex.simplex_rule(8)
    v = np.array([[1.0, 0.0], [math.cos(0.3), math.sin(0.3)], [0.8, 0.1]])
    _, J = simplex.blended_map(v, simplex.circle_arc(0, 0, 1, 0.0, 0.3), xi, eta)
    chord = 0.5 * abs((v[1, 0] - v[0, 0]) * (v[2, 1] - v[0, 1]) - (v[2, 0] - v[0, 0]) * (v[1, 1] - v[0, 1]))
    segment = 0.5 * (0.3 - math.sin(0.3))
    assert abs(np.sum(w * J) - (chord + segment)) < 1e-14


def test_disk_mesh_is_a_quadrature_rule_for_the_disk():
    m = meshes.disk_mesh(base_level=4, fine_level=5, centres=[[0.2, 0.1]], refine_radius={5: 0.2})
    assert abs(m.w.sum() - math.pi) < 1e-13
    assert np.all(m.w > 0) and np.max(np.hypot(m.xy[:, 0], m.xy[:, 1])) < 1.0
    # far field of a radial density: -(1/2pi) log|r0| times the mass (Gauss's law)
    sigma = 0.1
    f = inputs.f_disk(m.xy[:, 0], m.xy[:, 1], sigma)
    mass = math.pi + math.pi * sigma**2 * (1 - math.exp(-1 / sigma**2))
    tgt = np.array([[2.0, 0.5], [-1.5, -1.5]])
    V = oracle.evaluate(m.xy, m.w, f, tgt)
    ref = -np.log(np.hypot(tgt[:, 0], tgt[:, 1])) * mass / (2 * math.pi)
    assert np.max(np.abs(V - ref)) < 1e-10
