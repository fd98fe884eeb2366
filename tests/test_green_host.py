"""The host Green functions of libvp (vp_green_eval_host: the Bessel routines
the modified-Helmholtz plans use for their operator tables) against scipy and
mpmath. Host code only; no GPU needed."""

import math

import numpy as np
import pytest
from scipy.special import kv


def test_green_eval_host_matches_scipy_and_mpmath():
    from paper_2203_05933_gb300 import vp

    for lam in (0.5, 10.0, 300.0):
        r = np.geomspace(1e-9, 2.0, 4001) / min(lam, 1.0)
        r = r[lam * r < 650.0]
        g = vp.green_eval_host(r, vp.VP_KERNEL_MHELMHOLTZ, lam)
        ref = lam * lam / (2 * math.pi) * kv(0, lam * r)
        assert np.max(np.abs(g - ref) / ref) < 2e-14
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for x in (1e-6, 0.37, 1.999, 2.001, 7.5, 40.0, 200.0):
        g = vp.green_eval_host(np.array([x / 10.0]), vp.VP_KERNEL_MHELMHOLTZ, 10.0)[0]
        ref = float(100 / (2 * mp.pi) * mp.besselk(0, x))
        assert abs(g - ref) <= 2e-15 * abs(ref) * 8
    lg = vp.green_eval_host(np.array([0.5, 2.0]), vp.VP_KERNEL_LAPLACE)
    assert np.allclose(lg, -np.log([0.5, 2.0]) / (2 * math.pi), rtol=1e-15)
    with pytest.raises(vp.VPError):
        vp.green_eval_host(np.array([0.0]), vp.VP_KERNEL_MHELMHOLTZ, 1.0)
    with pytest.raises(vp.VPError):
        vp.green_eval_host(np.array([1.0]), vp.VP_KERNEL_MHELMHOLTZ, -1.0)
