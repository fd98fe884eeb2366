"""Oversampling set-up (host, untimed): interpolation matrices, the collapsed
triangle rule, and box corrections taken against the oversampled smooth rule,
pinned against exact polynomial values, exact moments and the closed-form
potential of f = 1 on a square."""

import math

import numpy as np
import scipy.sparse as sp

import oracle
from paper_2203_05933_gb300 import inputs
from paper_2203_05933_gb300.setup import corrections as C
from paper_2203_05933_gb300.setup import simplex
from paper_2203_05933_gb300.setup import upsample as U
from test_oracle_pins import rect_potential


def test_box_interpolation_reproduces_polynomials():
    L = U.box_upsample_1d(8, 16)
    xp, _ = np.polynomial.legendre.leggauss(8)
    xq, _ = np.polynomial.legendre.leggauss(16)
    for k in range(8):
        assert np.max(np.abs(L @ xp**k - xq**k)) < 1e-13
    assert np.max(np.abs(L @ xp**8 - xq**8)) > 1e-6  # degree p is not reproduced
    # two-dimensional: Kronecker product on y-major, x-fastest node order
    X, Y = np.meshgrid(xp, xp, indexing="xy")
    Xq, Yq = np.meshgrid(xq, xq, indexing="xy")
    f = X.ravel() ** 3 * Y.ravel() ** 6 + X.ravel() ** 7
    fq = np.kron(L, L) @ f
    assert np.max(np.abs(fq - (Xq.ravel() ** 3 * Yq.ravel() ** 6 + Xq.ravel() ** 7))) < 1e-13


def test_collapsed_rule_moments():
    xi, eta, w = U.collapsed_triangle_rule(9)
    assert np.all(w > 0) and xi.size == 81
    for a in range(17):
        for b in range(17 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * xi**a * eta**b) - exact) < 1e-15, (a, b)


def test_triangle_interpolation_reproduces_polynomials():
    xi_q, eta_q, _ = U.collapsed_triangle_rule(9)
    O = U.triangle_upsample(8, xi_q, eta_q)
    xi_p, eta_p, _ = simplex.simplex_rule(8)
    for a, b in [(0, 0), (1, 0), (0, 1), (3, 4), (7, 0), (2, 5)]:
        assert np.max(np.abs(O @ (xi_p**a * eta_p**b) - xi_q**a * eta_q**b)) < 1e-11, (a, b)


def test_oversampled_rule_with_corrections_is_exact_for_constant_density():
    nbox = 4
    p = inputs.box_grid_problem(nbox=nbox, order=8, csr="none")
    xq, wq, ups = U.box_grid_upsampled(nbox, 8, 16)
    ref = np.array([rect_potential(x, y, -1, 1, -1, 1) for x, y in p.tgt_xy])
    f1 = np.ones((1, p.n_src))
    smooth_q = oracle.evaluate(xq, wq, U.apply(ups, f1), p.tgt_xy, None)[0]
    smooth_p = oracle.evaluate(p.src_xy, p.w, f1, p.tgt_xy, None)[0]
    e_q, e_p = np.max(np.abs(smooth_q - ref)), np.max(np.abs(smooth_p - ref))
    assert e_q < e_p / 10  # oversampling shrinks the smooth rule's near-field error
    csr = C.box_grid_csr(nbox, 8, q=16)
    M = sp.csr_matrix((csr[2], csr[1], csr[0]), shape=(p.n_tgt, p.n_src))
    assert np.max(np.abs(smooth_q + M @ f1[0] - ref)) < 1e-12
    # a polynomial of degree 7 in each variable: oracle with corrections against
    # the same polynomial's potential from the area-to-line basis potentials
    fpoly = (p.src_xy[:, 0] ** 3 * p.src_xy[:, 1] ** 2 + p.src_xy[:, 1] ** 7)[None, :]
    V = oracle.evaluate(xq, wq, U.apply(ups, fpoly), p.tgt_xy, None)[0] + M @ fpoly[0]
    Vp = oracle.evaluate(p.src_xy, p.w, fpoly, p.tgt_xy, C.box_grid_csr(nbox, 8))[0]
    assert np.max(np.abs(V - Vp)) < 1e-12
