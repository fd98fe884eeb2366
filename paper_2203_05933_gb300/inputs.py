"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws and lays out inputs: quadrature nodes and weights of
the cells, source densities, target points and the sparsity pattern (and, for
parity-only runs, seeded values) of the correction matrix. It holds none of the
volume-potential arithmetic, so both the CUDA path and the CPU oracle can take
their inputs from here.

Layout conventions (the ones the C ABI uses):
  * points are float64 arrays of shape [n, 2] holding (x, y);
  * densities are float64 arrays of shape [ndens, n_src];
  * the correction matrix is CSR (rowptr int64 [n_tgt + 1], col int32, val
    float64), rows indexed by targets, columns by source nodes.

Workloads mirror the cells of the paper: regular boxes carrying tensor
Gauss-Legendre nodes (the box cells of Sec. 4.2, here with Gauss-Legendre in
place of Chebyshev roots), and seeded point clouds for ragged cases.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2203_05933


@dataclass
class Problem:
    """One volume-potential evaluation problem in caller order."""

    name: str
    src_xy: np.ndarray  # [n_src, 2]
    w: np.ndarray  # [n_src]
    tgt_xy: np.ndarray  # [n_tgt, 2]
    f: np.ndarray  # [ndens, n_src]
    csr: tuple | None = None  # (rowptr, col, val)
    root: tuple | None = None  # (x0, y0, side) of the enclosing square, when known
    meta: dict = field(default_factory=dict)

    @property
    def n_src(self) -> int:
        return int(self.src_xy.shape[0])

    @property
    def n_tgt(self) -> int:
        return int(self.tgt_xy.shape[0])

    @property
    def ndens(self) -> int:
        return int(self.f.shape[0])

    @property
    def nnz(self) -> int:
        return 0 if self.csr is None else int(self.csr[0][-1])


def gauss_legendre(order: int):
    """Gauss-Legendre nodes and weights on [-1, 1] (numpy's routine)."""
    return np.polynomial.legendre.leggauss(order)


def box_grid_nodes(nbox: int, order: int, lo: float = -1.0, hi: float = 1.0):
    """Nodes and weights of an nbox x nbox grid of boxes, order x order tensor GL.

    Ordered cell by cell (cell index = by * nbox + bx), then node (iy, ix) inside
    the cell. Weights are w_GL(ix) w_GL(iy) (side / 2)^2, i.e. the reference
    weights times the constant Jacobian of the box map.
    Returns (xy [n, 2], w [n], cell [n]).
    """
    t, wt = gauss_legendre(order)
    side = (hi - lo) / nbox
    half = side / 2.0
    cx = lo + half + side * np.arange(nbox)
    by, bx, iy, ix = np.meshgrid(np.arange(nbox), np.arange(nbox), np.arange(order),
                                 np.arange(order), indexing="ij")
    x = cx[bx] + half * t[ix]
    y = cx[by] + half * t[iy]
    w = wt[ix] * wt[iy] * half * half
    cell = by * nbox + bx
    xy = np.stack([x.ravel(), y.ravel()], axis=1)
    return np.ascontiguousarray(xy), w.ravel().copy(), cell.ravel().copy()


def f_config1(x, y):
    """Source density of the 16x16-box workload: a Gaussian bump plus a smooth wave."""
    return np.exp(-25.0 * ((x - 0.1) ** 2 + (y + 0.2) ** 2)) + np.sin(3.0 * x) * np.cos(2.0 * y)


def neighbour_csr_pattern(nbox: int, order: int):
    """CSR pattern of the box-grid correction: each target node couples to every
    node of its own box and of the (up to) 8 boxes around it.
    Returns (rowptr int64, col int32)."""
    npc = order * order
    ncell = nbox * nbox
    cell_cols = []
    for by in range(nbox):
        for bx in range(nbox):
            cols = []
            for ny in range(max(0, by - 1), min(nbox, by + 2)):
                for nx in range(max(0, bx - 1), min(nbox, bx + 2)):
                    c = ny * nbox + nx
                    cols.append(np.arange(c * npc, (c + 1) * npc))
            cell_cols.append(np.concatenate(cols).astype(np.int32))
    lens = np.repeat(np.array([c.size for c in cell_cols], np.int64), npc)
    rowptr = np.zeros(ncell * npc + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    col = np.concatenate([np.tile(cell_cols[c], npc) for c in range(ncell)])
    return rowptr, col


def synthetic_csr_values(rowptr, col, w, seed: int, scale: float = 1.0):
    """Seeded stand-in values for a correction pattern, sized like real ones
    (a few times the node weight of the column). For parity and timing only."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(col.size)
    w = np.asarray(w)
    step = 1 << 26  # in place, a slice at a time (the matrices reach billions of entries)
    for a in range(0, col.size, step):
        v[a:a + step] *= w[col[a:a + step]]
    if scale != 1.0:
        v *= scale
    return v


def box_grid_problem(nbox: int = 16, order: int = 8, ndens: int = 1, seed: int = SEED_BASE + 1,
                     csr: str = "synthetic", name: str | None = None) -> Problem:
    """The uniform box-grid workload on [-1, 1]^2: sources = targets = the GL nodes.

    csr: "synthetic" (seeded values on the own + 8 neighbour pattern),
    "corrections" (the singular/near-singular corrections computed by the host
    set-up, setup.corrections.box_grid_csr), "none", or a (rowptr, col, val)
    tuple supplied by the caller.
    """
    xy, w, _ = box_grid_nodes(nbox, order)
    rng = np.random.default_rng(seed)
    f0 = f_config1(xy[:, 0], xy[:, 1])
    if ndens == 1:
        f = f0[None, :]
    else:
        f = np.vstack([f0[None, :], rng.standard_normal((ndens - 1, xy.shape[0]))])
    if isinstance(csr, tuple):
        mat = csr
    elif csr == "synthetic":
        rowptr, col = neighbour_csr_pattern(nbox, order)
        mat = (rowptr, col, synthetic_csr_values(rowptr, col, w, seed + 17))
    elif csr == "corrections":
        from .setup import corrections
        mat = corrections.box_grid_csr(nbox, order)
    else:
        mat = None
    return Problem(name=name or f"boxgrid{nbox}x{nbox}_gl{order}", src_xy=xy, w=w, tgt_xy=xy.copy(),
                   f=np.ascontiguousarray(f), csr=mat, root=(-1.0, -1.0, 2.0),
                   meta={"nbox": nbox, "order": order})


def random_csr(n_tgt: int, n_src: int, per_row_max: int, seed: int, empty_frac: float = 0.1):
    """Seeded random CSR with ragged rows (some empty), sorted columns."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, per_row_max + 1, size=n_tgt)
    lens[rng.random(n_tgt) < empty_frac] = 0
    lens = np.minimum(lens, n_src)
    rowptr = np.zeros(n_tgt + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    col = np.empty(int(rowptr[-1]), np.int32)
    for i in range(n_tgt):
        if lens[i]:
            col[rowptr[i]:rowptr[i + 1]] = np.sort(rng.choice(n_src, size=lens[i], replace=False))
    val = rng.standard_normal(col.size) * 1e-3
    return rowptr, col, val


def cloud_problem(n_src: int, n_tgt: int, ndens: int = 1, seed: int = SEED_BASE + 100,
                  shared: int = 0, clustered: bool = True, csr_per_row: int = 32,
                  name: str | None = None) -> Problem:
    """Seeded ragged point cloud: a mix of uniform points and Gaussian clusters in
    [-1, 1]^2, positive weights, Gaussian-mixture densities. The first `shared`
    targets coincide exactly with sources (the node-target case)."""
    rng = np.random.default_rng(seed)

    def pts(n):
        if not clustered:
            return rng.uniform(-1.0, 1.0, size=(n, 2))
        k = n // 2
        centres = rng.uniform(-0.7, 0.7, size=(5, 2))
        lab = rng.integers(0, 5, size=n - k)
        cl = centres[lab] + 0.03 * rng.standard_normal((n - k, 2))
        return np.clip(np.vstack([rng.uniform(-1.0, 1.0, size=(k, 2)), cl]), -0.999, 0.999)

    src = pts(n_src)
    tgt = pts(n_tgt)
    shared = min(shared, n_src, n_tgt)
    if shared:
        tgt[:shared] = src[rng.choice(n_src, size=shared, replace=False)]
    w = rng.uniform(0.5, 1.5, size=n_src) * 4.0 / n_src
    f = np.empty((ndens, n_src))
    for d in range(ndens):
        c = rng.uniform(-0.8, 0.8, size=(3, 2))
        a = rng.standard_normal(3)
        s = rng.uniform(0.05, 0.4, size=3)
        f[d] = sum(a[m] * np.exp(-((src[:, 0] - c[m, 0]) ** 2 + (src[:, 1] - c[m, 1]) ** 2) / s[m] ** 2)
                   for m in range(3)) + 0.1
    mat = random_csr(n_tgt, n_src, csr_per_row, seed + 1) if csr_per_row > 0 else None
    return Problem(name=name or f"cloud{n_src}x{n_tgt}", src_xy=np.ascontiguousarray(src), w=w,
                   tgt_xy=np.ascontiguousarray(tgt), f=f, csr=mat)


def normaliser(problem: Problem) -> np.ndarray:
    """sum_j |w_j f_j^d| per density: the scale of the relative l-infinity error."""
    return np.abs(problem.w[None, :] * problem.f).sum(axis=1)


def disk_centres(seed: int, k: int = 5, rmax: float = 0.8):
    """k seeded bump centres, uniform in the disk r < rmax."""
    rng = np.random.default_rng(seed)
    r = rmax * np.sqrt(rng.random(k))
    th = 2 * np.pi * rng.random(k)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def f_disk(x, y, sigma: float = 0.1):
    """Radial density 1 + exp(-r^2 / sigma^2) on the unit disk."""
    return 1.0 + np.exp(-(x * x + y * y) / sigma**2)


def disk_problem(base_level: int = 7, fine_level: int = 9, refine_radius=None, ndens: int = 1,
                 seed: int = SEED_BASE + 2, csr: str = "synthetic", name: str | None = None) -> Problem:
    """The unit-disk workload: quadtree boxes (8x8 Gauss-Legendre) refined around
    5 seeded bump centres, plus a band of curved and straight degree-7 triangles
    (36 nodes each); sources = targets = the nodes. With the defaults (levels
    7..9) it has about 1.1 M nodes. The correction pattern is self + near cells;
    its values are seeded stand-ins (parity and timing only)."""
    from .setup import meshes

    if refine_radius is None:
        refine_radius = {base_level + 1: 0.11, base_level + 2: 0.04}
    mesh = meshes.disk_mesh(base_level=base_level, fine_level=fine_level, centres=disk_centres(seed),
                            refine_radius=refine_radius)
    xy, w = mesh.xy, mesh.w
    f0 = f_disk(xy[:, 0], xy[:, 1])
    if ndens == 1:
        f = f0[None, :]
    else:
        rng = np.random.default_rng(seed + 3)
        f = np.empty((ndens, xy.shape[0]))
        f[0] = f0
        for d in range(1, ndens):  # random Gaussian mixtures
            c = rng.uniform(-0.7, 0.7, size=(4, 2))
            a = rng.standard_normal(4)
            s = rng.uniform(0.05, 0.5, size=4)
            f[d] = sum(a[m] * np.exp(-((xy[:, 0] - c[m, 0]) ** 2 + (xy[:, 1] - c[m, 1]) ** 2) / s[m] ** 2)
                       for m in range(4))
    mat = None
    if csr == "synthetic":
        rowptr, col = meshes.near_cell_pattern(mesh)
        mat = (rowptr, col, synthetic_csr_values(rowptr, col, w, seed + 17))
    return Problem(name=name or f"disk_L{base_level}-{fine_level}", src_xy=xy, w=w, tgt_xy=xy.copy(),
                   f=np.ascontiguousarray(f), csr=mat, root=(-1.0, -1.0, 2.0),
                   meta={"n_cells": mesh.ncell, "n_triangles": int((mesh.cell_kind > 0).sum()),
                         "base_level": base_level, "fine_level": fine_level})


def disk_upsampling(base_level: int = 7, fine_level: int = 9, refine_radius=None, seed: int = SEED_BASE + 2,
                    q_box: int = 16, m_tri: int = 9):
    """q-nodes of the disk workload's cells for the oversampled smooth rule
    (q = 2p: 16 x 16 Gauss-Legendre per box; collapsed Gauss rule with
    m_tri^2 nodes per triangle) and the per-cell interpolation from the p-nodes
    of disk_problem with the same arguments. Returns (xy_q, w_q, Upsampling)."""
    from .setup import meshes, upsample

    if refine_radius is None:
        refine_radius = {base_level + 1: 0.11, base_level + 2: 0.04}
    cen = disk_centres(seed)
    mp = meshes.disk_mesh(base_level=base_level, fine_level=fine_level, centres=cen, refine_radius=refine_radius)
    rule = upsample.collapsed_triangle_rule(m_tri)
    mq = meshes.disk_mesh(base_level=base_level, fine_level=fine_level, centres=cen, refine_radius=refine_radius,
                          box_order=q_box, tri_rule=rule)
    return mq.xy, mq.w, upsample.mesh_upsampling(mp, mq, 8, q_box, 8, rule)


def own_cell_csr(cell_start, w, seed: int):
    """Correction pattern that couples every node to the nodes of its own cell
    (block diagonal), with seeded stand-in values."""
    cell_start = np.asarray(cell_start, np.int64)
    sizes = np.diff(cell_start)
    rowptr = np.zeros(cell_start[-1] + 1, np.int64)
    np.cumsum(np.repeat(sizes, sizes), out=rowptr[1:])
    col = np.concatenate([np.tile(np.arange(a, b, dtype=np.int32), b - a)
                          for a, b in zip(cell_start[:-1], cell_start[1:])])
    return rowptr, col, synthetic_csr_values(rowptr, col, w, seed)


def many_problems(count: int = 256, n_min: int = 2048, n_max: int = 65536, seed: int = SEED_BASE + 4) -> list[Problem]:
    """Independent problems of uneven size for the many-problem batch: half box
    grids on squares (nbox x nbox boxes, 8x8 GL), half unit-disk meshes (boxes +
    curved triangle band), sizes log-uniform in [n_min, n_max] (box grids
    exactly, disks from three mesh levels); each problem scaled and shifted at
    random. Disk meshes are built once per level and reused (a similarity
    transform of a quadrature rule is a rule, with weights scaled by the square
    of the scale). The correction couples each node to its own cell (block
    diagonal, seeded values), which keeps the batch's host inputs small."""
    from .setup import meshes

    rng = np.random.default_rng(seed)
    disk_cache = {}
    out = []
    for i in range(count):
        target_n = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        scale = float(np.exp(rng.uniform(np.log(0.5), np.log(4.0))))
        shift = rng.uniform(-5.0, 5.0, size=2)
        if i % 2 == 0:
            nbox = int(np.clip(round(np.sqrt(target_n / 64.0)), 6, 32))
            xy, w, cell = box_grid_nodes(nbox, 8)
            cs = np.arange(0, xy.shape[0] + 1, 64, dtype=np.int64)
            kind = "square"
        else:
            base = int(np.clip(round(np.log(target_n / 3000.0) / np.log(4.0)) + 3, 3, 5))
            if base not in disk_cache:
                disk_cache[base] = meshes.disk_mesh(base_level=base, fine_level=base)
            m = disk_cache[base]
            xy, w, cs = m.xy, m.w, m.cell_start
            kind = "disk"
        xy = xy * scale + shift
        w = w * scale * scale
        f = np.exp(-((xy[:, 0] - shift[0]) ** 2 + (xy[:, 1] - shift[1]) ** 2) / (0.3 * scale) ** 2)[None, :] + 0.5
        root = (float(shift[0] - scale), float(shift[1] - scale), float(2.0 * scale))
        out.append(Problem(name=f"{kind}{i}", src_xy=np.ascontiguousarray(xy), w=w, tgt_xy=np.ascontiguousarray(xy),
                           f=np.ascontiguousarray(f), csr=own_cell_csr(cs, w, seed + 1000 + i), root=root,
                           meta={"kind": kind}))
    return out


# ---------------------------------------------------------------------------
# Star domain with holes: r(theta) = 1 + 0.3 cos(5 theta), 12 circular holes
# ---------------------------------------------------------------------------

STAR_SIZES = {
    # name: (base box level, refinement radius in Gaussian widths, total targets)
    "4M": (8, 41.0, 1 << 22),
    "1M": (7, 14.0, 1 << 20),
    "small": (7, 0.0, 1 << 14),
}


def star_geometry(seed: int = SEED_BASE + 3, count: int = 50):
    """Holes (rows cx, cy, R; radii uniform in [0.02, 0.08], gaps >= 0.12) and the
    Gaussians of the density (centres uniform in the domain, widths log-uniform
    in [1e-3, 1e-1], amplitudes N(0, 1))."""
    from .setup import meshes

    holes = meshes.star_holes(seed, gap=0.12)
    rng = np.random.default_rng(seed + 1)
    cen = []
    while len(cen) < count:
        p = rng.uniform(-1.3, 1.3, size=2)
        if meshes.inside_star(np.array([p[0]]), np.array([p[1]]), holes)[0]:
            cen.append(p)
    width = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), size=count))
    amp = rng.standard_normal(count)
    return holes, np.array(cen), width, amp


def f_star(x, y, centres, width, amp):
    """Sum of Gaussians a_i exp(-|r - c_i|^2 / s_i^2)."""
    out = np.zeros_like(x)
    for (cx, cy), s, a in zip(centres, width, amp):
        out += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (s * s))
    return out


def star_random_points(n: int, holes, seed: int):
    """n seeded points uniform in the star minus its holes (rejection sampling)."""
    from .setup import meshes

    rng = np.random.default_rng(seed)
    out = [np.zeros((0, 2))]
    have = 0
    while have < n:
        p = rng.uniform(-1.3, 1.3, size=(max(2 * (n - have), 1024), 2))
        p = p[meshes.inside_star(p[:, 0], p[:, 1], holes)]
        out.append(p)
        have += p.shape[0]
    return np.ascontiguousarray(np.vstack(out)[:n])


def cell_rows_csr(cell_start, tgt_cell, cell_cols=None):
    """CSR whose row i holds the columns of cell tgt_cell[i]: the nodes of that
    cell itself (cell_cols None), or cell_cols[c], the column list of cell c.
    Returns (rowptr int64, col int32)."""
    cell_start = np.asarray(cell_start, np.int64)
    tgt_cell = np.asarray(tgt_cell, np.int64)
    if cell_cols is None:
        lens = np.diff(cell_start)[tgt_cell]
        rowptr = np.zeros(tgt_cell.size + 1, np.int64)
        np.cumsum(lens, out=rowptr[1:])
        col = (np.repeat(cell_start[tgt_cell] - rowptr[:-1], lens) + np.arange(rowptr[-1])).astype(np.int32)
        return rowptr, col
    lens = np.array([cell_cols[c].size for c in tgt_cell], np.int64)
    rowptr = np.zeros(tgt_cell.size + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    col = np.empty(int(rowptr[-1]), np.int32)
    for i, c in enumerate(tgt_cell):
        col[rowptr[i]:rowptr[i + 1]] = cell_cols[c]
    return rowptr, col


def star_problem(size: str = "4M", ndens: int = 1, seed: int = SEED_BASE + 3, targets: str = "mixed",
                 csr: str = "own", extra_targets=None, name: str | None = None) -> Problem:
    """The star-with-holes workload: quadtree boxes (8x8 Gauss-Legendre) of a
    base level, refined towards the narrow Gaussians of the density (a box of
    side b is split while b > 2 s_i and it lies within rho s_i of centre c_i),
    plus bands of curved and straight degree-7 triangles (36 nodes) along the
    star boundary and around the holes.

    size: "4M" (about 4.1 M nodes, 2^22 targets), "1M" (about 1 M nodes, 2^20
    targets) or "small" (unrefined level-7 boxes, 2^14 targets).
    targets: "mixed" (a seeded subsample of the nodes, at most half of them and
    of the total, plus uniform random interior points up to the total) or "nodes" (targets = sources).
    csr: "own" (each target couples to the nodes of its cell; a random target
    to those of the cell whose centre is nearest), "near" (the cells touching
    that cell as well), or "none"; values are seeded stand-ins.
    extra_targets: optional [k, 2] points appended to the targets (no
    correction rows)."""
    from .setup import meshes

    base, rho, total = STAR_SIZES[size]
    holes, cen, width, amp = star_geometry(seed)

    def refine(level, x0, y0, b):
        d = meshes._box_point_dist(x0, y0, b, cen[:, 0], cen[:, 1])
        return bool(np.any((b > 2.0 * width) & (d < rho * width)))

    mesh = meshes.star_mesh(holes, base_level=base, fine_level=11, refine=refine if rho > 0 else None)
    xy, w = mesh.xy, mesh.w
    f0 = f_star(xy[:, 0], xy[:, 1], cen, width, amp)
    if ndens == 1:
        f = f0[None, :]
    else:
        rng = np.random.default_rng(seed + 3)
        f = np.empty((ndens, xy.shape[0]))
        f[0] = f0
        for d in range(1, ndens):
            c = rng.uniform(-0.9, 0.9, size=(4, 2))
            a = rng.standard_normal(4)
            s = rng.uniform(0.05, 0.5, size=4)
            f[d] = f_star(xy[:, 0], xy[:, 1], c, s, a)
    node_cell = np.repeat(np.arange(mesh.ncell), np.diff(mesh.cell_start))
    if targets == "nodes":
        tgt = xy.copy()
        tgt_cell = node_cell
    else:
        rng = np.random.default_rng(seed + 5)
        n_sub = min(xy.shape[0] // 2, total // 2)
        sub = np.sort(rng.choice(xy.shape[0], size=n_sub, replace=False))
        rnd = star_random_points(total - n_sub, holes, seed + 6)
        from scipy.spatial import cKDTree

        bb = mesh.cell_bbox
        cc = np.stack([(bb[:, 0] + bb[:, 1]) / 2, (bb[:, 2] + bb[:, 3]) / 2], axis=1)
        _, near = cKDTree(cc).query(rnd)
        # the random points are stored cell by cell (stable order within a cell),
        # so that the correction rows of one cell are consecutive
        order = np.argsort(near, kind="stable")
        rnd, near = rnd[order], near[order]
        tgt = np.ascontiguousarray(np.vstack([xy[sub], rnd]))
        tgt_cell = np.concatenate([node_cell[sub], near])
    mat = None
    if csr in ("own", "near"):
        cols = None
        if csr == "near":
            cols = meshes.near_cell_columns(mesh)
        rowptr, col = cell_rows_csr(mesh.cell_start, tgt_cell, cols)
        mat = (rowptr, col, synthetic_csr_values(rowptr, col, w, seed + 17))
    if extra_targets is not None:
        tgt = np.ascontiguousarray(np.vstack([tgt, np.asarray(extra_targets, float).reshape(-1, 2)]))
        if mat is not None:
            k = tgt.shape[0] - (mat[0].size - 1)
            mat = (np.concatenate([mat[0], np.full(k, mat[0][-1], np.int64)]), mat[1], mat[2])
    return Problem(name=name or f"star_{size}", src_xy=xy, w=w, tgt_xy=tgt, f=np.ascontiguousarray(f), csr=mat,
                   root=(-1.3, -1.3, 2.6),
                   meta={"n_cells": mesh.ncell, "n_triangles": int((mesh.cell_kind > 0).sum()), "holes": holes,
                         "area": mesh.area, "base_level": base})
