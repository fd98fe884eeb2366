"""Triangle self-correction blocks generated on the GPU (vp_tricorr) against
the plain host evaluation of the same fixed rule
(setup.tricorr.self_corrections_reference) for straight, circle-arc and
polar-arc (star) cells."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05933_gb300 import inputs, vp  # noqa: E402
from paper_2203_05933_gb300.setup import meshes, tricorr  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()


def _check(mesh, cells, tc, R):
    geom = np.array([tricorr.geom_params(mesh.geom[k]) for k in cells])
    out = tc.eval(geom).cpu().numpy()
    worst = 0.0
    for i, k in enumerate(cells):
        ref = tricorr.self_corrections_reference(mesh.geom[k], R)
        worst = max(worst, float(np.max(np.abs(out[i] - ref)) / np.max(np.abs(ref))))
    return worst


def test_disk_triangles_match_host_rule():
    R = tricorr.self_rules(8)
    tc = vp.TriCorr(R)
    m = meshes.disk_mesh(base_level=4, fine_level=5, centres=[[0.1, 0.2]], refine_radius={5: 0.2})
    tris = [k for k, g in enumerate(m.geom) if g[0] == "tri"]
    err = _check(m, tris[:40], tc, R)
    print(f"disk triangles: GPU vs host rule max rel diff {err:.2e}")
    assert err < 1e-12
    tc.close()


def test_star_triangles_match_host_rule():
    R = tricorr.self_rules(8)
    tc = vp.TriCorr(R)
    holes, _, _, _ = inputs.star_geometry()
    m = meshes.star_mesh(holes, base_level=7, fine_level=7)
    kinds = {}
    for k, g in enumerate(m.geom):
        if g[0] == "tri":
            key = 0 if g[2] is None else int(g[2].spec[0])
            kinds.setdefault(key, []).append(k)
    cells = kinds[0][:8] + kinds[1][:8] + kinds[2][:8]
    err = _check(m, cells, tc, R)
    print(f"star triangles (straight, hole arcs, star arcs): max rel diff {err:.2e}")
    assert err < 1e-12
    tc.close()


def test_tricorr_bad_arguments_raise():
    R = tricorr.self_rules(8)
    bad = dict(R)
    bad["tau"] = R["tau"].copy()
    bad["tau"][0, 0] = 0.0
    with pytest.raises(vp.VPError):
        vp.TriCorr(bad)
