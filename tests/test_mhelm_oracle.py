"""Pins of the modified-Helmholtz oracle (oracle/mhelm.py) against facts that
do not come from the oracle itself.

The kernel is G(r, r0) = (lambda^2 / 2 pi) K0(lambda |r - r0|) (arXiv
2203.05933, Sec. 2). A dropped lambda^2, K0(r) in place of K0(lambda r), another
Bessel function, a transposed adjoint or a coincident pair that is not skipped
each fails one of the checks below.
"""

import math

import numpy as np
import pytest
from scipy.special import iv, kv

from oracle import mhelm
from paper_2203_05933_gb300 import inputs


@pytest.mark.parametrize("lam", [1.0, 3.0])
def test_disk_exterior_closed_form(lam):
    # Graf's addition theorem integrated over the disk |r| < R with f = 1: only the
    # n = 0 term survives the angular integral, so outside the disk
    # V(r0) = (lambda^2/2pi) K0(lambda|r0|) 2pi int_0^R I0(lambda rho) rho drho
    #       = lambda R I1(lambda R) K0(lambda |r0|).
    pr = inputs.disk_problem(base_level=4, fine_level=4, csr=None)
    th = np.linspace(0.1, 2 * np.pi + 0.1, 9, endpoint=False)
    for rad in (1.8, 2.0, 2.5):
        tg = np.stack([rad * np.cos(th), rad * np.sin(th)], axis=1)
        v = mhelm.evaluate(pr.src_xy, pr.w, np.ones(pr.n_src), tg, lam)[0]
        exact = lam * iv(1, lam) * kv(0, lam * rad)
        assert np.max(np.abs(v - exact)) / exact < 1e-10


def test_tiny_brute_force_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    lam = 2.5
    src = np.array([[0.1, 0.2], [-0.3, 0.05], [0.25, -0.4]])
    w = np.array([0.7, 1.1, 0.4])
    f = np.array([[1.5, -0.5, 2.0]])
    tgt = np.array([[0.0, 0.0], [0.1, 0.2], [0.9, 0.3]])  # the second coincides with source 0
    got = mhelm.evaluate(src, w, f, tgt, lam)[0]
    for i in range(3):
        s = mp.mpf(0)
        for j in range(3):
            r = mp.sqrt((mp.mpf(tgt[i, 0]) - src[j, 0]) ** 2 + (mp.mpf(tgt[i, 1]) - src[j, 1]) ** 2)
            if r == 0:
                continue
            s += mp.mpf(w[j]) * f[0, j] * lam**2 / (2 * mp.pi) * mp.besselk(0, lam * r)
        assert abs(got[i] - float(s)) <= 1e-14 * abs(float(s))


def test_exterior_modified_helmholtz_equation():
    # away from the sources V solves -Delta V + lambda^2 V = 0 (fourth-order
    # differences); log or K1 kernels, or K0 at the wrong scale, do not
    rng = np.random.default_rng(5)
    lam = 4.0
    src = rng.uniform(-0.3, 0.3, size=(40, 2))
    w = rng.uniform(0.5, 1.0, size=40)
    f = rng.standard_normal((1, 40))
    h = 2e-3
    for x0, y0 in ((0.9, 0.1), (-0.2, 0.8)):
        st = [(0, 0)] + [(k * h, 0) for k in (-2, -1, 1, 2)] + [(0, k * h) for k in (-2, -1, 1, 2)]
        pts = np.array([[x0 + a, y0 + b] for a, b in st])
        v = mhelm.evaluate(src, w, f, pts, lam)[0]
        c = np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / (12.0 * h * h)
        lap = c @ np.array([v[1], v[2], v[0], v[3], v[4]]) + c @ np.array([v[5], v[6], v[0], v[7], v[8]])
        res = -lap + lam * lam * v[0]
        assert abs(res) < 1e-6 * lam * lam * abs(v[0])
        assert abs(lap) > 1e-2 * lam * lam * abs(v[0])  # the check is not vacuous


def test_adjoint_identity_and_correction():
    prob = inputs.cloud_problem(300, 250, ndens=2, shared=40, seed=41, csr_per_row=6)
    lam = 6.0
    g = np.random.default_rng(2).standard_normal((2, prob.n_tgt))
    Af = mhelm.evaluate(prob.src_xy, prob.w, prob.f, prob.tgt_xy, lam, prob.csr)
    ATg = mhelm.adjoint(prob.src_xy, prob.w, g, prob.tgt_xy, lam, prob.csr)
    for d in range(2):
        lhs, rhs = float(g[d] @ Af[d]), float(ATg[d] @ prob.f[d])
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1e-300) * 10
    # the correction term is exactly the CSR product, written out entry by entry
    plain = mhelm.evaluate(prob.src_xy, prob.w, prob.f, prob.tgt_xy, lam)
    rowptr, col, val = prob.csr
    for i in range(0, prob.n_tgt, 17):
        s = sum(val[k] * prob.f[0, col[k]] for k in range(rowptr[i], rowptr[i + 1]))
        assert abs(Af[0, i] - plain[0, i] - s) <= 1e-12 * (abs(s) + abs(plain[0, i]))
    # sampled sources of the adjoint agree with the full one
    cols = np.arange(0, prob.n_src, 29)
    subc = mhelm.adjoint_cols(prob.src_xy, prob.w, g, prob.tgt_xy, cols, lam, prob.csr)
    assert np.allclose(subc, ATg[:, cols], rtol=1e-13, atol=1e-13 * np.abs(ATg).max())
    # sampled rows agree with the full evaluation
    rows = np.arange(0, prob.n_tgt, 23)
    sub = mhelm.evaluate_rows(prob.src_xy, prob.w, prob.f, prob.tgt_xy, rows, lam, prob.csr)
    assert np.allclose(sub, Af[:, rows], rtol=1e-13, atol=1e-13 * np.abs(Af).max())


def test_coincident_pair_skipped():
    lam = 3.0
    src = np.array([[0.0, 0.0], [0.5, 0.0]])
    w = np.array([1.0, 1.0])
    f = np.array([[1.0, 1.0]])
    v = mhelm.evaluate(src, w, f, src, lam)[0]
    g = lam * lam / (2 * math.pi) * kv(0, lam * 0.5)
    assert abs(v[0] - g) < 1e-15 and abs(v[1] - g) < 1e-15
