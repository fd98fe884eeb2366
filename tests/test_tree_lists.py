"""Host-side checks of the adaptive quadtree and its interaction lists (no GPU).

The FMM is exact in its bookkeeping only if every (source, target) pair is
counted exactly once: directly (U), through a multipole evaluated at the target
(W), a multipole-to-local translation between ancestors (V), or a source-to-local
expansion (X). These tests check that partition on ragged adaptive trees, plus
the geometric separation each far-field list relies on.
"""

import numpy as np
import pytest

from paper_2203_05933_gb300 import inputs, vp


@pytest.fixture(scope="module")
def lib():
    from paper_2203_05933_gb300 import build
    build.build()
    return vp._load()


def _ancestors(parent, b):
    out = []
    while b >= 0:
        out.append(b)
        b = parent[b]
    return out


def _csr_sets(ptr, idx):
    return [set(idx[ptr[b]:ptr[b + 1]].tolist()) for b in range(len(ptr) - 1)]


def _adjacent(lvl, ixy, a, b):
    L = max(lvl[a], lvl[b])
    sa, sb = 1 << (L - lvl[a]), 1 << (L - lvl[b])
    ax0, ay0 = ixy[a] * sa
    bx0, by0 = ixy[b] * sb
    return ax0 <= bx0 + sb and bx0 <= ax0 + sa and ay0 <= by0 + sb and by0 <= ay0 + sa


@pytest.mark.parametrize("n_src,n_tgt,leaf,seed", [(2500, 2000, 16, 1), (1200, 1500, 8, 2), (3000, 0, 32, 3)])
def test_every_pair_counted_once(lib, n_src, n_tgt, leaf, seed):
    p = inputs.cloud_problem(n_src, max(n_tgt, 1), seed=seed, shared=min(n_tgt, 300), csr_per_row=0)
    tgt = p.tgt_xy if n_tgt else p.src_xy
    t = vp.vp_tree_build(p.src_xy, tgt, vp.make_options(leaf=leaf))
    lvl, ixy, parent, is_leaf = t["box_level"], t["box_ixy"], t["box_parent"], t["box_leaf"]
    U, V = _csr_sets(t["u_ptr"], t["u_idx"]), _csr_sets(t["v_ptr"], t["v_idx"])
    W, X = _csr_sets(t["w_ptr"], t["w_idx"]), _csr_sets(t["x_ptr"], t["x_idx"])
    leaves = np.nonzero(is_leaf)[0]
    assert len(leaves) > 20 and lvl.max() >= 4  # a genuinely adaptive tree
    anc = {b: _ancestors(parent, b) for b in leaves}
    for B in leaves:
        ancB = anc[B]
        for A in leaves:
            ancA = set(anc[A])
            c = int(A in U[B])
            c += sum(1 for D in W[B] if D in ancA)
            c += sum(1 for Bp in ancB for C in V[Bp] if C in ancA)
            c += sum(1 for Bp in ancB if A in X[Bp])
            assert c == 1, (B, A, c)


def test_list_geometry(lib):
    p = inputs.cloud_problem(3000, 2000, seed=4, csr_per_row=0)
    t = vp.vp_tree_build(p.src_xy, p.tgt_xy, vp.make_options(leaf=12))
    lvl, ixy, parent, is_leaf = t["box_level"], t["box_ixy"], t["box_parent"], t["box_leaf"]
    V = _csr_sets(t["v_ptr"], t["v_idx"])
    W = _csr_sets(t["w_ptr"], t["w_idx"])
    X = _csr_sets(t["x_ptr"], t["x_idx"])
    for b, vb in enumerate(V):
        for c in vb:
            assert lvl[c] == lvl[b]
            off = np.abs(ixy[c] - ixy[b])
            assert off.max() >= 2 and off.max() <= 3  # well separated, within the parent's neighbours
            assert _adjacent(lvl, ixy, parent[c], parent[b])
    for b, wb in enumerate(W):
        if wb:
            assert is_leaf[b]
        for d in wb:
            assert not _adjacent(lvl, ixy, d, b) and _adjacent(lvl, ixy, parent[d], b)
            assert lvl[d] > lvl[b]
            assert b in X[d]


def test_points_partitioned_by_leaves(lib):
    p = inputs.cloud_problem(4000, 3000, seed=5, csr_per_row=0)
    opts = vp.make_options(leaf=20)
    t = vp.vp_tree_build(p.src_xy, p.tgt_xy, opts)
    assert sorted(t["src_perm"].tolist()) == list(range(4000))
    assert sorted(t["tgt_perm"].tolist()) == list(range(3000))
    is_leaf = t["box_leaf"].astype(bool)
    for rng, n in ((t["box_src"], 4000), (t["box_tgt"], 3000)):
        cover = np.zeros(n, int)
        for b0, b1 in rng[is_leaf]:
            cover[b0:b1] += 1
        assert np.all(cover == 1)
        assert np.all(rng[is_leaf][:, 1] - rng[is_leaf][:, 0] <= 20) or t["box_level"].max() == 24


def test_points_inside_their_leaf_box(lib):
    p = inputs.box_grid_problem(nbox=6, order=8, csr="none")
    opts = vp.make_options(leaf=64, root=(-1.0, -1.0, 2.0))
    t = vp.vp_tree_build(p.src_xy, p.tgt_xy, opts)
    lvl, ixy = t["box_level"], t["box_ixy"]
    pts = p.src_xy[t["src_perm"]]
    for b in np.nonzero(t["box_leaf"])[0]:
        side = 2.0 / (1 << lvl[b])
        lo = -1.0 + ixy[b] * side
        s0, s1 = t["box_src"][b]
        q = pts[s0:s1]
        assert np.all(q >= lo) and np.all(q < lo + side)


def test_tree_rejects_bad_input(lib):
    xy = np.array([[0.0, 0.0], [np.nan, 1.0]])
    with pytest.raises(vp.VPError):
        vp.vp_tree_build(xy, xy)
    with pytest.raises(vp.VPError):
        vp.vp_tree_build(np.array([[2.0, 0.0]]), np.array([[0.0, 0.0]]),
                         vp.make_options(root=(-1.0, -1.0, 2.0)))
    with pytest.raises(vp.VPError):
        vp.vp_tree_build(np.zeros((4, 2)), np.zeros((4, 2)), vp.make_options(leaf=100000))


def test_coincident_points_stop_at_max_level(lib):
    xy = np.zeros((200, 2))
    xy[100:] = 0.5
    t = vp.vp_tree_build(xy, xy, vp.make_options(leaf=8, max_level=6))
    assert t["box_level"].max() <= 6
