"""The float64 near field's own logarithm, measured through the public API.

One source at the origin with unit weight and density and targets on the x axis
at multiples of 2^-50 (so that their coordinates are exact on the integer grid
the directed near field uses, and r^2 = dx^2 is formed exactly there, then
rounded once to 53 bits): with a single leaf every pair is summed directly, the
local expansion is zero, and out_i = -(1/2pi) * (1/2) log(r_i^2) up to the
final multiplication. So |out - ref| measures the logarithm's own error. The
table-driven method (Tang 1990: table spacing 2^-12, cubic log1p, e log 2 and
the table logarithm added in float64) has absolute error below
2^-52 max(1, |e| log 2) plus half an ulp of the result (e the binary exponent
of r^2), plus 2^-53 for the rounding of r^2 (the reference rounds r^2 too):
about one ulp of log r^2 where |log r^2| >= 1. The coincident pair gives 0.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05933_gb300 import vp  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()


def test_log64_within_three_ulp():
    rng = np.random.default_rng(5)
    # log-uniform distances over 1e-12 .. 40,
    # plus values next to powers of two and table points, where the rounding of
    # the table index changes
    r = np.exp(rng.uniform(np.log(1e-12), np.log(40.0), 3000))
    p2 = np.ldexp(1.0, np.arange(-30, 5))
    near = np.concatenate([p2 * (1 + 1e-15), p2 * (1 - 1e-15), p2 * (1 + 2.0 ** -13), p2 * (1 - 2.0 ** -14)])
    r = np.concatenate([r, np.sqrt(near)])
    r = np.round(np.ldexp(r, 50)) * 2.0 ** -50  # on the grid: exact integer coordinates
    n = r.size
    tgt = np.stack([r, np.zeros(n)], axis=1)
    tgt = np.vstack([tgt, [[0.0, 0.0]]])  # the coincident target: no smooth term
    src = np.zeros((1, 2))
    w = np.ones(1)
    plan = vp.Plan.create(src, w, tgt, None, p_fmm=16, leaf=4096, root=(-64.0, -64.0, 128.0))
    assert plan.info().n_leaves == 1
    out = plan.eval(torch.ones((1, 1), dtype=torch.float64, device="cuda")).cpu().numpy()[0]
    inv2pi = 0.159154943091895335768883763372514362
    r2 = r * r
    L = np.log(r2)
    ref = -inv2pi * (0.5 * L)
    e = np.frexp(r2)[1] - 1
    bound = 0.5 * inv2pi * (2.0 ** -52 * np.maximum(1.0, np.abs(e) * np.log(2.0)) + 2.0 ** -52
                            + np.spacing(np.abs(L))) + 2.0 * np.spacing(np.abs(ref))
    ratio = np.abs(out[:n] - ref) / bound
    big = np.abs(L) >= 1.0
    ulps = np.abs(out[:n] - ref)[big] / np.spacing(np.abs(ref[big]))
    print(f"log64: error / bound max {ratio.max():.3f}; where |log r^2| >= 1: max {ulps.max():.2f} ulp, "
          f"mean {ulps.mean():.3f} ulp over {big.sum()} distances")
    assert ratio.max() <= 1.0
    assert ulps.max() <= 3.0
    assert out[n] == 0.0
    plan.close()


def test_default_and_plain_kernels_agree_on_a_line():
    # the same line of targets through the plain FP64 kernels (CUDA's log): the
    # two results differ by at most the logarithm's error
    rng = np.random.default_rng(6)
    r = np.exp(rng.uniform(np.log(1e-6), np.log(4.0), 2000))
    r = np.round(np.ldexp(r, 50)) * 2.0 ** -50
    tgt = np.stack([r, np.zeros(r.size)], axis=1)
    outs = []
    for flags in (0, vp.VP_FLAG_FP64):
        plan = vp.Plan.create(np.zeros((1, 2)), np.ones(1), tgt, None, p_fmm=16, leaf=4096,
                              root=(-8.0, -8.0, 16.0), flags=flags)
        outs.append(plan.eval(torch.ones((1, 1), dtype=torch.float64, device="cuda")).cpu().numpy()[0])
        plan.close()
    inv2pi = 0.159154943091895335768883763372514362
    L = np.log(r * r)
    e = np.frexp(r * r)[1] - 1
    bound = 0.5 * inv2pi * (2.0 ** -52 * np.maximum(1.0, np.abs(e) * np.log(2.0)) + 2.0 ** -52
                            + 2 * np.spacing(np.abs(L))) + 2.0 * np.spacing(np.abs(outs[1]))
    assert np.max(np.abs(outs[0] - outs[1]) / bound) <= 1.0
