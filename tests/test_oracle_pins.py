"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each check would fail under a plausible mistake in the oracle: a dropped
-1/(2pi), log r^2 used as log r, a transposed operand, a missing correction
term, a sign error in the adjoint or in the target gradient, or a coincident
pair that is not skipped.
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.sparse

import oracle
from paper_2203_05933_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rect_antiderivative(x, y):
    """F with d2F/dxdy = log(x^2 + y^2) (checked symbolically below):
    F = x y log(x^2+y^2) - 3 x y + x^2 atan(y/x) + y^2 atan(x/y), with the
    x = 0 / y = 0 limits (the atan terms vanish there)."""
    x = np.asarray(x, float)
    y = np.asarray(y, float)
    r2 = x * x + y * y
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = np.where(r2 > 0, x * y * np.log(np.where(r2 > 0, r2, 1.0)), 0.0)
        t3 = np.where(x != 0, x * x * np.arctan(y / np.where(x != 0, x, 1.0)), 0.0)
        t4 = np.where(y != 0, y * y * np.arctan(x / np.where(y != 0, y, 1.0)), 0.0)
    return t1 - 3.0 * x * y + t3 + t4


def rect_potential(x0, y0, a, b, c, d):
    """Exact volume potential of f = 1 on [a,b]x[c,d] at (x0, y0):
    -(1/4pi) * int int log((x-x0)^2 + (y-y0)^2) dx dy, by the corner rule."""
    F = rect_antiderivative
    s = (F(b - x0, d - y0) - F(a - x0, d - y0) - F(b - x0, c - y0) + F(a - x0, c - y0))
    return -s / (4.0 * math.pi)


def test_rect_antiderivative_symbolic():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y", positive=True)
    F = x * y * sympy.log(x**2 + y**2) - 3 * x * y + x**2 * sympy.atan(y / x) + y**2 * sympy.atan(x / y)
    assert sympy.simplify(sympy.diff(F, x, y) - sympy.log(x**2 + y**2)) == 0


@pytest.mark.parametrize("pt", [(0.0, 3.0), (2.5, 0.3), (-1.7, 2.2)])
def test_rect_closed_form_against_adaptive_quadrature(pt):
    # the closed form itself, checked against scipy's adaptive 2-D quadrature
    x0, y0 = pt
    ref, _ = scipy.integrate.dblquad(
        lambda y, x: -math.log((x - x0) ** 2 + (y - y0) ** 2) / (4 * math.pi),
        -1.0, 1.0, -1.0, 1.0, epsabs=1e-14, epsrel=1e-14)
    assert abs(rect_potential(x0, y0, -1, 1, -1, 1) - ref) < 1e-12


def test_oracle_rectangle_far_targets():
    # f = 1 on [-1,1]^2 through the smooth rule (4x4 boxes, 16x16 GL): at targets
    # well outside the square the rule is spectrally accurate, so the oracle's
    # point sum must reproduce the closed form.
    xy, w, _ = inputs.box_grid_nodes(4, 16)
    tgt = np.array([[0.0, 3.0], [2.5, 0.3], [-1.7, 2.2], [3.0, -3.0], [-2.0, -1.5]])
    got = oracle.evaluate(xy, w, np.ones(xy.shape[0]), tgt)
    ref = np.array([rect_potential(x, y, -1, 1, -1, 1) for x, y in tgt])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_oracle_disk_far_targets():
    # radial density on the unit disk through a polar product rule; outside the
    # disk the potential is -(1/2pi) log|r0| times the total mass (Gauss's law
    # for the logarithmic kernel)
    sigma = 0.3
    nr, nt = 48, 96
    tr, wr = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * (tr + 1.0)
    wr = 0.5 * wr
    th = 2 * np.pi * np.arange(nt) / nt
    R, TH = np.meshgrid(r, th, indexing="ij")
    xy = np.stack([(R * np.cos(TH)).ravel(), (R * np.sin(TH)).ravel()], axis=1)
    w = (np.outer(wr * r, np.full(nt, 2 * np.pi / nt))).ravel()
    f = 1.0 + np.exp(-(R.ravel() ** 2) / sigma**2)
    mass = np.pi + np.pi * sigma**2 * (1 - math.exp(-1 / sigma**2))
    tgt = np.array([[1.5, 0.0], [0.0, -2.0], [2.0, 2.0], [-1.2, 0.9]])
    got = oracle.evaluate(xy, w, f, tgt)
    ref = -np.log(np.hypot(tgt[:, 0], tgt[:, 1])) * mass / (2 * np.pi)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_oracle_tiny_hand_values():
    with open(os.path.join(GOLDEN, "tiny_hand.json")) as fh:
        case = json.load(fh)
    env = {"log": math.log, "sqrt": math.sqrt, "pi": math.pi, "__builtins__": {}}
    ref = np.array([eval(e, env) for e in case["expected_formula"]])
    got = oracle.evaluate(np.array(case["sources"]), np.array(case["weights"]),
                          np.array(case["density"]), np.array(case["targets"]))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)


def _dense_reference(p):
    # independent brute force: dense kernel matrix (numpy) + scipy sparse CSR
    d = p.tgt_xy[:, None, :] - p.src_xy[None, :, :]
    r = np.hypot(d[..., 0], d[..., 1])
    coincident = (d[..., 0] == 0) & (d[..., 1] == 0)
    with np.errstate(divide="ignore"):
        G = np.where(coincident, 0.0, -np.log(np.where(coincident, 1.0, r)) / (2 * np.pi))
    V = (G @ (p.w[None, :] * p.f).T).T
    if p.csr is not None:
        rowptr, col, val = p.csr
        P = scipy.sparse.csr_matrix((val, col, rowptr), shape=(p.n_tgt, p.n_src))
        V = V + (P @ p.f.T).T
    return V, G


def test_oracle_matches_dense_brute_force():
    p = inputs.cloud_problem(700, 500, ndens=3, shared=120, seed=11)
    ref, _ = _dense_reference(p)
    got = oracle.evaluate(p.src_xy, p.w, p.f, p.tgt_xy, p.csr)
    scale = inputs.normaliser(p)[:, None]
    assert np.max(np.abs(got - ref) / scale) < 1e-14


def test_oracle_csr_term_is_the_sparse_product():
    p = inputs.cloud_problem(300, 200, ndens=2, seed=12)
    with_c = oracle.evaluate(p.src_xy, p.w, p.f, p.tgt_xy, p.csr)
    without = oracle.evaluate(p.src_xy, p.w, p.f, p.tgt_xy, None)
    rowptr, col, val = p.csr
    P = scipy.sparse.csr_matrix((val, col, rowptr), shape=(p.n_tgt, p.n_src))
    np.testing.assert_allclose(with_c - without, (P @ p.f.T).T, rtol=0, atol=1e-15)


def test_oracle_adjoint_dot_product_and_dense():
    p = inputs.cloud_problem(400, 350, ndens=2, shared=80, seed=13)
    rng = np.random.default_rng(5)
    g = rng.standard_normal((2, p.n_tgt))
    Af = oracle.evaluate(p.src_xy, p.w, p.f, p.tgt_xy, p.csr)
    Atg = oracle.adjoint(p.src_xy, p.w, g, p.tgt_xy, p.csr)
    lhs = np.sum(Af * g, axis=1)
    rhs = np.sum(p.f * Atg, axis=1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)
    # against the transposed dense matrix
    _, G = _dense_reference(p)
    rowptr, col, val = p.csr
    P = scipy.sparse.csr_matrix((val, col, rowptr), shape=(p.n_tgt, p.n_src))
    ref = (p.w[:, None] * (G.T @ g.T)).T + (P.T @ g.T).T
    np.testing.assert_allclose(Atg, ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def test_oracle_target_gradient_finite_differences():
    p = inputs.cloud_problem(300, 60, ndens=2, seed=14, csr_per_row=8)
    # keep targets at least 2e-2 away from every source so that central FD is accurate
    d = np.hypot(*(p.tgt_xy[:, None, :] - p.src_xy[None, :, :]).transpose(2, 0, 1))
    keep = d.min(axis=1) > 2e-2
    tgt = p.tgt_xy[keep]
    rows = np.nonzero(keep)[0]
    csr = oracle.csr_rows(p.csr, rows)
    rng = np.random.default_rng(6)
    g = rng.standard_normal((2, tgt.shape[0]))
    grad = oracle.grad_targets(p.src_xy, p.w, p.f, g, tgt)
    h = 1e-6
    for k in range(2):
        e = np.zeros_like(tgt)
        e[:, k] = h
        Vp = oracle.evaluate(p.src_xy, p.w, p.f, tgt + e, csr)
        Vm = oracle.evaluate(p.src_xy, p.w, p.f, tgt - e, csr)
        fd = np.sum(g * (Vp - Vm), axis=0) / (2 * h)
        np.testing.assert_allclose(grad[:, k], fd, rtol=1e-6, atol=1e-8)


def test_oracle_coincident_pair_excluded_and_near_pair_kept():
    src = np.array([[0.25, 0.5], [0.25 + 1e-9, 0.5]])
    w = np.array([1.0, 1.0])
    f = np.array([1.0, 1.0])
    got = oracle.evaluate(src, w, f, np.array([[0.25, 0.5]]))
    gap = src[1, 0] - src[0, 0]  # the representable separation, about 1e-9
    assert abs(got[0] - (-math.log(gap) / (2 * math.pi))) < 1e-14


def test_oracle_threads_do_not_change_result():
    p = inputs.cloud_problem(500, 400, ndens=2, seed=15)
    a = oracle.evaluate(p.src_xy, p.w, p.f, p.tgt_xy, p.csr, nthreads=1)
    b = oracle.evaluate(p.src_xy, p.w, p.f, p.tgt_xy, p.csr, nthreads=4)
    assert np.array_equal(a, b)


def test_oracle_grad_scale_bounds_and_closed_forms():
    # one source: the normaliser is |g q| / (2 pi r) = |dL/dt|; sources on a ray on
    # one side with charges of one sign: every term points the same way, so the
    # normaliser equals |dL/dt|; random clouds: it bounds |dL/dt| from above
    t = np.array([[0.3, -0.2]])
    s = np.array([[1.1, 0.4]])
    r = np.hypot(0.8, 0.6)
    sc = oracle.grad_scale(s, np.array([0.7]), np.array([[2.0]]), np.array([[-1.5]]), t)
    assert abs(sc[0] - 1.5 * 0.7 * 2.0 / (2 * np.pi * r)) <= 1e-15
    ray = np.array([[0.3 + a, -0.2] for a in (0.1, 0.25, 0.7, 1.3)])
    w = np.array([0.5, 1.0, 2.0, 0.25])
    f = np.array([[1.0, 3.0, 0.5, 2.0]])
    g = np.array([[0.8]])
    sc = oracle.grad_scale(ray, w, f, g, t)
    gr = oracle.grad_targets(ray, w, f, g, t)
    assert abs(sc[0] - np.hypot(*gr[0])) <= 1e-14 * sc[0]
    rng = np.random.default_rng(9)
    src = rng.uniform(-1, 1, (300, 2))
    tgt = np.vstack([rng.uniform(-1, 1, (40, 2)), src[:5]])  # some coincident targets
    w = rng.uniform(0.1, 1.0, 300)
    f = rng.standard_normal((2, 300))
    g = rng.standard_normal((2, 45))
    sc = oracle.grad_scale(src, w, f, g, tgt)
    gr = oracle.grad_targets(src, w, f, g, tgt)
    assert np.all(np.hypot(gr[:, 0], gr[:, 1]) <= sc * (1 + 1e-13))
    # the brute-force definition written out with numpy
    d = np.hypot(tgt[:, None, 0] - src[None, :, 0], tgt[:, None, 1] - src[None, :, 1])
    with np.errstate(divide="ignore"):
        inv = np.where(d > 0, 1.0 / d, 0.0)
    want = np.einsum("di,dj,ij->i", np.abs(g), np.abs(w[None, :] * f), inv) / (2 * np.pi)
    assert np.max(np.abs(sc - want) / want) <= 1e-13
