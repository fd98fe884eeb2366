"""The correction apply of float64 plans (exact fixed-point sums: each row's
values as integers of at most 52 bits under one power of two, the group's
densities likewise, 128-bit totals rounded once) against the exactly rounded
sum of the float64 products (math.fsum), on a matrix built to stress the
fixed-point form: rows whose values span 300 orders of magnitude, rows of one
scale from 1e-150 to 1e150, zero and empty rows, densities spanning 60 orders
of magnitude with zeros among them, column lists from 1 to 3500 columns (the
longest beyond the staging buffer, so it takes the float64 loop).

The bound per row follows from the representation: the values are rounded to
2^-53 of the power of two above the row's largest one (at most 2^-52 of it),
the densities likewise against the group's largest, the reference's own
products to 2^-53 each, the result once more; rows beyond the staging buffer
add the float64 loop's summation error. The FMM part is made
negligible (weights 1e-250), so the plan's output is the correction product."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05933_gb300 import vp  # noqa: E402

U = 2.0 ** -53
STAGED_MAX = 3072  # longer column lists take the float64 loop


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()


def _problem(seed=11, n_src=5000):
    rng = np.random.default_rng(seed)
    src = rng.uniform(-1, 1, (n_src, 2))
    rowptr, cols, vals, lens = [0], [], [], []
    sizes = [1, 2, 3, 37, 200, 576, 1448, 3500]
    kinds = ["narrow", "wide", "tiny", "huge", "zero"]
    while len(lens) < 3000:
        m = int(rng.choice(sizes)) if rng.random() > 0.03 else 0
        c = rng.choice(n_src, size=m, replace=False).astype(np.int32)
        for _ in range(int(rng.integers(1, 24))):  # rows of one group share the columns
            kind = kinds[int(rng.integers(len(kinds)))]
            sign = rng.choice([-1.0, 1.0], size=m)
            if kind == "narrow":
                v = sign * rng.uniform(0.01, 1.0, m)
            elif kind == "wide":
                v = sign * 10.0 ** rng.uniform(-150, 150, m)
            elif kind == "tiny":
                v = sign * 10.0 ** rng.uniform(-152, -148, m)
            elif kind == "huge":
                v = sign * 10.0 ** rng.uniform(148, 152, m)
            else:
                v = np.zeros(m)
            cols.append(c)
            vals.append(v)
            lens.append(m)
            rowptr.append(rowptr[-1] + m)
    n_tgt = len(lens)
    tgt = rng.uniform(-1, 1, (n_tgt, 2))
    csr = (np.array(rowptr, np.int64), np.concatenate(cols).astype(np.int32), np.concatenate(vals))
    return src, tgt, csr


def _densities(rng, nd, n):
    f = rng.choice([-1.0, 1.0], size=(nd, n)) * 10.0 ** rng.uniform(-30, 30, (nd, n))
    f[rng.random((nd, n)) < 0.02] = 0.0
    return f


def _check_rows(out, f, csr, what):
    rowptr, col, val = csr
    worst = 0.0
    for r in range(rowptr.size - 1):
        a, b = rowptr[r], rowptr[r + 1]
        v, c = val[a:b], col[a:b]
        for d in range(f.shape[0]):
            x = f[d, c]
            prod = v * x
            ref = math.fsum(prod)
            vmax = float(np.max(np.abs(v))) if b > a else 0.0
            xmax = float(np.max(np.abs(x))) if b > a else 0.0
            bound = (2 * U * vmax * float(np.sum(np.abs(x))) + 2 * U * xmax * float(np.sum(np.abs(v)))
                     + U * float(np.sum(np.abs(prod))) + 2 * U * abs(ref))
            if b - a > STAGED_MAX:
                bound += (b - a) * U * float(np.sum(np.abs(prod)))
            err = abs(float(out[d, r]) - ref)
            assert err <= 2 * bound + 1e-200, (what, r, d, b - a, err, bound, ref)
            if bound > 0:
                worst = max(worst, err / bound)
    print(f"{what}: largest error over its bound {worst:.3f}")


@pytest.mark.parametrize("nd", [1, 2, 4, 8])
def test_fixed_point_apply_matches_exact_sums(nd):
    src, tgt, csr = _problem()
    rng = np.random.default_rng(20 + nd)
    f = _densities(rng, nd, src.shape[0])
    w = np.full(src.shape[0], 1e-250)
    plan = vp.Plan.create(src, w, tgt, csr, p_fmm=16, leaf=64, max_dens=8)
    out = plan.eval(torch.as_tensor(f, device="cuda")).cpu().numpy()
    _check_rows(out, f, csr, f"forward, {nd} densities")
    # the same call again: the staging and the sums start from nothing each time
    out2 = plan.eval(torch.as_tensor(f, device="cuda")).cpu().numpy()
    assert np.array_equal(out, out2)
    plan.close()


def test_fixed_point_adjoint_matches_exact_sums():
    # Pi^T g from the stored values (each converted back to float64 exactly):
    # the values' rounding (2^-52 of the row's largest) plus float64 summation
    src, tgt, csr = _problem(seed=12)
    rowptr, col, val = csr
    rng = np.random.default_rng(31)
    # moderate magnitudes: the row scale is applied to g, which must stay normal
    keep = np.abs(val) > 0
    val = np.where(keep, np.sign(val) * np.clip(np.abs(val), 1e-100, 1e100), 0.0)
    csr = (rowptr, col, val)
    g = rng.standard_normal((1, tgt.shape[0]))
    w = np.full(src.shape[0], 1e-250)
    plan = vp.Plan.create(src, w, tgt, csr, p_fmm=16, leaf=64)
    gf = plan.adjoint(torch.as_tensor(g, device="cuda"))[0].cpu().numpy()[0]
    rows = np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr))
    prod = val * g[0, rows]
    n_src = src.shape[0]
    vmax_row = np.zeros(rowptr.size - 1)
    np.maximum.at(vmax_row, rows, np.abs(val))
    order = np.argsort(col, kind="stable")
    starts = np.searchsorted(col[order], np.arange(n_src + 1))
    worst = 0.0
    for j in range(n_src):
        idx = order[starts[j]:starts[j + 1]]
        ref = math.fsum(prod[idx])
        s_abs = float(np.sum(np.abs(prod[idx])))
        q = 2 * U * float(np.sum(vmax_row[rows[idx]] * np.abs(g[0, rows[idx]])))
        bound = q + (idx.size + 2) * U * s_abs
        err = abs(gf[j] - ref)
        assert err <= 2 * bound + 1e-200, (j, err, bound)
        if bound > 0:
            worst = max(worst, err / bound)
    print(f"adjoint: largest error over its bound {worst:.3f}")
    plan.close()
