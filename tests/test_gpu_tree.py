"""The tree and interaction lists built on the GPU (vp_tree_build_device, what
vp_plan_create uses) equal the host build (vp_tree_build, checked on CPU in
test_tree_lists.py) array by array: box levels, coordinates, parents,
children, leaf flags, point ranges, both permutations and the U/V/W/X lists."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2203_05933_gb300 import inputs, vp  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05933_gb300 import build
    build.build()


def _compare(src, tgt, **opts):
    o = vp.make_options(**opts)
    h = vp.vp_tree_build(src, tgt, o)
    d = vp.vp_tree_build_device(src, tgt, o)
    assert h.keys() == d.keys()
    for k in h:
        assert h[k].shape == d[k].shape, k
        assert np.array_equal(h[k], d[k]), k
    return h


@pytest.mark.parametrize("leaf", [1, 8, 32, 64, 128])
def test_cloud_trees_match(leaf):
    p = inputs.cloud_problem(5000, 4000, shared=1500, seed=90 + leaf, csr_per_row=0)
    h = _compare(p.src_xy, p.tgt_xy, leaf=leaf)
    assert len(h["box_level"]) > 1


def test_coincident_points_and_level_cap():
    # many points at the same coordinates: equal keys keep caller order; the
    # level cap stops the splitting
    rng = np.random.default_rng(3)
    xy = rng.uniform(-1, 1, (3000, 2))
    xy[1000:2000] = xy[5]
    xy[2000:2300] = [0.25, -0.5]
    _compare(xy, xy[::-1].copy(), leaf=16, max_level=6)
    _compare(xy, xy, leaf=4, max_level=20)


def test_given_root_and_empty_sets():
    rng = np.random.default_rng(4)
    s = rng.uniform(0, 1, (2000, 2))
    _compare(s, np.zeros((0, 2)), leaf=32, root=(0.0, 0.0, 1.0))
    _compare(np.zeros((0, 2)), s, leaf=32)
    _compare(s, s + 1e-9, leaf=32, root=(-0.5, -0.5, 2.0))


def test_mesh_trees_match():
    disk = inputs.disk_problem(base_level=5, fine_level=7)
    _compare(disk.src_xy, disk.tgt_xy, leaf=64, root=disk.root)
    _compare(disk.src_xy, disk.tgt_xy, leaf=128)
    star = inputs.star_problem("small", csr="none")
    _compare(star.src_xy, star.tgt_xy, leaf=64, root=star.root)


def test_star_4M_tree_matches():
    star = inputs.star_problem("4M", csr="none")
    h = _compare(star.src_xy, star.tgt_xy, leaf=64, root=star.root)
    assert len(h["box_level"]) > 100000
