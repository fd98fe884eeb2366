"""Synthetic domain decompositions of the kind the paper meshes (Sec. 3.1):
regular boxes in the bulk (here an adaptive quadtree refined around seeded
bumps) and a thin band of boundary-fitted curved triangles plus straight
triangles between the boxes and the boundary, with the quadrature nodes and
weights of every cell (Jacobians folded in, Eq. vio_rokh_quad_rule and the box
rule of Sec. 4.2).

Stand-ins, stated once: the paper's band comes from Gmsh after a buffer zone of
delta*h (Sec. 3.1); here boxes are kept when they lie inside r <= 1 - delta*h
and the gap to the circle is cut into radial strips, one per edge of the
staircase boundary of the kept boxes (that boundary is star-shaped about the
centre, so the radial cuts do not cross it), each strip split into one curved
and one straight triangle.
Triangles whose outer edge is a circle arc use the blending map of
Eq. deformed_triangle_maps; the others are affine.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import simplex


@dataclass
class Mesh:
    xy: np.ndarray          # [n, 2] quadrature nodes, cell by cell (triangles first, then boxes)
    w: np.ndarray           # [n] weights (reference weight x Jacobian)
    cell_start: np.ndarray  # [ncell + 1] node range of each cell
    cell_bbox: np.ndarray   # [ncell, 4] xmin, xmax, ymin, ymax
    cell_kind: np.ndarray   # [ncell] 0 box, 1 straight triangle, 2 curved triangle
    cell_level: np.ndarray  # [ncell] quadtree level for boxes, -1 for triangles
    area: float             # exact area of the domain

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])

    @property
    def ncell(self) -> int:
        return int(self.cell_kind.size)


def _box_dist(x0, y0, side, c):
    dx = max(x0 - c[0], 0.0, c[0] - (x0 + side))
    dy = max(y0 - c[1], 0.0, c[1] - (y0 + side))
    return math.hypot(dx, dy)


def _staircase_loop(adm: np.ndarray):
    """Boundary of the union of admitted cells of an n x n grid as a closed
    counter-clockwise loop of integer lattice vertices (every lattice point on
    the boundary, so each loop edge is one cell side).
    adm[i, j] refers to cell column i (x) and row j (y)."""
    n = adm.shape[0]
    nxt = {}

    def a(i, j):
        return 0 <= i < n and 0 <= j < n and adm[i, j]

    for i, j in zip(*np.nonzero(adm)):
        # directed edges with the cell on the left (counter-clockwise)
        if not a(i, j - 1):
            nxt[(i, j)] = (i + 1, j)
        if not a(i + 1, j):
            nxt[(i + 1, j)] = (i + 1, j + 1)
        if not a(i, j + 1):
            nxt[(i + 1, j + 1)] = (i, j + 1)
        if not a(i - 1, j):
            nxt[(i, j + 1)] = (i, j)
    start = next(iter(nxt))
    loop = [start]
    v = nxt[start]
    while v != start:
        loop.append(v)
        v = nxt[v]
    if len(loop) != len(nxt):
        raise RuntimeError("admitted cells do not form one simply connected region")
    return np.array(loop)


def disk_mesh(base_level: int = 7, fine_level: int = 9, centres=None, refine_radius=None,
              delta: float = 0.8, box_order: int = 8, tri_p: int = 8) -> Mesh:
    """Unit disk: quadtree boxes over [-1, 1]^2 at `base_level` inside
    r <= 1 - delta*h, refined towards `fine_level` near the given centres
    (refine a level-l box into level l+1 while it lies within refine_radius[l+1]
    of a centre), plus the triangle band. Box nodes: box_order^2 tensor
    Gauss-Legendre; triangle nodes: tri_p (tri_p+1)/2 simplex nodes."""
    centres = np.zeros((0, 2)) if centres is None else np.asarray(centres, float)
    refine_radius = refine_radius or {}
    n = 1 << base_level
    h = 2.0 / n
    edges = -1.0 + h * np.arange(n + 1)
    X0, Y0 = np.meshgrid(edges[:-1], edges[:-1], indexing="ij")
    far = np.maximum(np.maximum(np.hypot(X0, Y0), np.hypot(X0 + h, Y0)),
                     np.maximum(np.hypot(X0, Y0 + h), np.hypot(X0 + h, Y0 + h)))
    adm = far <= 1.0 - delta * h

    # boxes with refinement
    boxes = []  # (level, x0, y0, side)
    stack = [(base_level, float(X0[i, j]), float(Y0[i, j]), h) for i, j in zip(*np.nonzero(adm))]
    while stack:
        lvl, x0, y0, side = stack.pop()
        r = refine_radius.get(lvl + 1, 0.0)
        if lvl < fine_level and centres.size and min(_box_dist(x0, y0, side, c) for c in centres) < r:
            s2 = side / 2
            stack.extend([(lvl + 1, x0, y0, s2), (lvl + 1, x0 + s2, y0, s2), (lvl + 1, x0, y0 + s2, s2),
                          (lvl + 1, x0 + s2, y0 + s2, s2)])
        else:
            boxes.append((lvl, x0, y0, side))
    boxes.sort(key=lambda b: (b[0], b[2], b[1]))

    # triangle band: radial strips between consecutive staircase vertices and
    # their projections onto the circle, each split into a curved and a
    # straight triangle along the diagonal that gives the larger minimum angle
    inner = _staircase_loop(adm).astype(float) * h - 1.0
    ang = np.arctan2(inner[:, 1], inner[:, 0])
    order = np.argsort(ang)
    inner, ang = inner[order], ang[order]
    if np.any(np.diff(ang) <= 0):
        raise RuntimeError("staircase is not strictly star-shaped about the centre")
    outer = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    m = inner.shape[0]

    def orient(a, b, c):
        return (b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1])

    def min_angle(a, b, c):
        out = []
        for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
            u, v = q - p, r - p
            out.append(math.acos(np.clip(np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v)), -1, 1)))
        return min(out)

    tris = []  # (kind, vertices[3,2], (th0, th1) for curved)
    for j in range(m):
        j1 = (j + 1) % m
        th0 = ang[j]
        th1 = ang[j1] + (2 * math.pi if j1 == 0 else 0.0)
        Ij, Ij1, Oj, Oj1 = inner[j], inner[j1], outer[j], outer[j1]
        splits = [((Oj, Oj1, Ij), (Ij, Ij1, Oj1)), ((Oj, Oj1, Ij1), (Oj, Ij1, Ij))]
        best = None
        for c_tri, s_tri in splits:
            if orient(*c_tri) <= 0 or orient(*s_tri) <= 0:
                continue
            q = min(min_angle(*c_tri), min_angle(*s_tri))
            if best is None or q > best[0]:
                best = (q, c_tri, s_tri)
        if best is None:
            raise RuntimeError("no valid split of a band strip")
        tris.append((2, np.array(best[1]), (th0, th1)))
        tris.append((1, np.array(best[2]), None))

    txi, teta, tw = simplex.simplex_rule(tri_p)
    bx, by, bw = simplex.gauss_legendre_box(box_order)
    xs, ws, start, bbox, kind, level = [], [], [0], [], [], []
    for k, v, th in tris:
        if k == 2:
            pts, J = simplex.blended_map(v, simplex.circle_arc(0.0, 0.0, 1.0, th[0], th[1]), txi, teta)
            lo_th, hi_th = th
            arc_x = np.cos(np.linspace(lo_th, hi_th, 9))
            arc_y = np.sin(np.linspace(lo_th, hi_th, 9))
            bb = [min(v[:, 0].min(), arc_x.min()), max(v[:, 0].max(), arc_x.max()),
                  min(v[:, 1].min(), arc_y.min()), max(v[:, 1].max(), arc_y.max())]
        else:
            pts, J = simplex.affine_map(v, txi, teta)
            bb = [v[:, 0].min(), v[:, 0].max(), v[:, 1].min(), v[:, 1].max()]
        if np.any(J <= 0):
            raise RuntimeError("degenerate triangle in the band")
        xs.append(pts)
        ws.append(tw * J)
        start.append(start[-1] + pts.shape[0])
        bbox.append(bb)
        kind.append(k)
        level.append(-1)
    for lvl, x0, y0, side in boxes:
        half = side / 2
        xs.append(np.stack([x0 + half + half * bx, y0 + half + half * by], axis=1))
        ws.append(bw * half * half)
        start.append(start[-1] + bx.size)
        bbox.append([x0, x0 + side, y0, y0 + side])
        kind.append(0)
        level.append(lvl)
    return Mesh(xy=np.ascontiguousarray(np.vstack(xs)), w=np.concatenate(ws),
                cell_start=np.array(start, np.int64), cell_bbox=np.array(bbox), cell_kind=np.array(kind, np.int8),
                cell_level=np.array(level, np.int32), area=math.pi)


def near_cell_pattern(mesh: Mesh, tol: float = 1e-9):
    """CSR pattern of a correction matrix: every node of a cell couples to every
    node of each cell whose bounding box touches or overlaps its own (the cell
    itself included) -- the self + near cells of the separation rule (Sec. 3.1).
    Returns (rowptr int64, col int32)."""
    from scipy.spatial import cKDTree

    bb = mesh.cell_bbox
    cen = np.stack([(bb[:, 0] + bb[:, 1]) / 2, (bb[:, 2] + bb[:, 3]) / 2], axis=1)
    half = np.stack([(bb[:, 1] - bb[:, 0]) / 2, (bb[:, 3] - bb[:, 2]) / 2], axis=1)
    reach = float(np.max(np.hypot(half[:, 0], half[:, 1]))) * 2 + tol
    tree = cKDTree(cen)
    cand = tree.query_ball_point(cen, r=reach)
    cs = mesh.cell_start
    cols, lens = [], []
    for k in range(mesh.ncell):
        c = np.array(cand[k])
        ov = ((np.abs(cen[c, 0] - cen[k, 0]) <= half[c, 0] + half[k, 0] + tol)
              & (np.abs(cen[c, 1] - cen[k, 1]) <= half[c, 1] + half[k, 1] + tol))
        nb = np.sort(c[ov])
        ck = np.concatenate([np.arange(cs[m], cs[m + 1]) for m in nb]).astype(np.int32)
        nk = int(cs[k + 1] - cs[k])
        cols.append(np.tile(ck, nk))
        lens.append(np.full(nk, ck.size, np.int64))
    lens = np.concatenate(lens)
    rowptr = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    return rowptr, np.concatenate(cols)
