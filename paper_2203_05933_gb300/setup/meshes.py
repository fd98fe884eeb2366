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
    geom: list | None = None  # per cell: ("box", x0, y0, side) or ("tri", vertices [3, 2], curve or None)

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
              delta: float = 0.8, box_order: int = 8, tri_p: int = 8, tri_rule=None) -> Mesh:
    """Unit disk: quadtree boxes over [-1, 1]^2 at `base_level` inside
    r <= 1 - delta*h, refined towards `fine_level` near the given centres
    (refine a level-l box into level l+1 while it lies within refine_radius[l+1]
    of a centre), plus the triangle band. Box nodes: box_order^2 tensor
    Gauss-Legendre; triangle nodes: tri_p (tri_p+1)/2 simplex nodes, or the
    given rule tri_rule = (xi, eta, w) on the reference triangle."""
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

    txi, teta, tw = simplex.simplex_rule(tri_p) if tri_rule is None else tri_rule
    bx, by, bw = simplex.gauss_legendre_box(box_order)
    xs, ws, start, bbox, kind, level = [], [], [0], [], [], []
    geom = []
    for k, v, th in tris:
        geom.append(("tri", v, simplex.circle_arc(0.0, 0.0, 1.0, th[0], th[1]) if k == 2 else None))
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
        geom.append(("box", x0, y0, side))
    return Mesh(xy=np.ascontiguousarray(np.vstack(xs)), w=np.concatenate(ws),
                cell_start=np.array(start, np.int64), cell_bbox=np.array(bbox), cell_kind=np.array(kind, np.int8),
                cell_level=np.array(level, np.int32), area=math.pi, geom=geom)


def near_cell_columns(mesh: Mesh, tol: float = 1e-9):
    """For each cell, the nodes (int32, ascending cell order) of every cell whose
    bounding box touches or overlaps its own, the cell itself included -- the
    self + near cells of the separation rule (Sec. 3.1)."""
    from scipy.spatial import cKDTree

    bb = mesh.cell_bbox
    cen = np.stack([(bb[:, 0] + bb[:, 1]) / 2, (bb[:, 2] + bb[:, 3]) / 2], axis=1)
    half = np.stack([(bb[:, 1] - bb[:, 0]) / 2, (bb[:, 3] - bb[:, 2]) / 2], axis=1)
    reach = float(np.max(np.hypot(half[:, 0], half[:, 1]))) * 2 + tol
    tree = cKDTree(cen)
    cand = tree.query_ball_point(cen, r=reach)
    cs = mesh.cell_start
    out = []
    for k in range(mesh.ncell):
        c = np.array(cand[k])
        ov = ((np.abs(cen[c, 0] - cen[k, 0]) <= half[c, 0] + half[k, 0] + tol)
              & (np.abs(cen[c, 1] - cen[k, 1]) <= half[c, 1] + half[k, 1] + tol))
        nb = np.sort(c[ov])
        out.append(np.concatenate([np.arange(cs[m], cs[m + 1]) for m in nb]).astype(np.int32))
    return out


def near_cell_pattern(mesh: Mesh, tol: float = 1e-9):
    """CSR pattern of a correction matrix: every node of a cell couples to every
    node of each cell whose bounding box touches or overlaps its own (the cell
    itself included). Returns (rowptr int64, col int32)."""
    cs = mesh.cell_start
    cols, lens = [], []
    for k, ck in enumerate(near_cell_columns(mesh, tol)):
        nk = int(cs[k + 1] - cs[k])
        cols.append(np.tile(ck, nk))
        lens.append(np.full(nk, ck.size, np.int64))
    lens = np.concatenate(lens)
    rowptr = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=rowptr[1:])
    return rowptr, np.concatenate(cols)


# ---------------------------------------------------------------------------
# Star-shaped domain with circular holes
# ---------------------------------------------------------------------------


def star_radius(theta, a: float = 0.3, k: int = 5):
    """Boundary r(theta) = 1 + a cos(k theta) and its derivative."""
    return 1.0 + a * np.cos(k * theta), -a * k * np.sin(k * theta)


def star_curve(th0, th1, a: float = 0.3, k: int = 5):
    """Arc of the star boundary from polar angle th0 to th1 as a curve on [0, 1]."""
    dth = th1 - th0

    def curve(s):
        th = th0 + s * dth
        r, dr = star_radius(th, a, k)
        c, sn = np.cos(th), np.sin(th)
        return r * c, r * sn, dth * (dr * c - r * sn), dth * (dr * sn + r * c)

    curve.spec = (2.0, a, float(k), th0, th1)
    return curve


def _staircase_loops(adm: np.ndarray):
    """Boundaries of the union of admitted cells of an n x n grid as closed
    loops of integer lattice vertices (every lattice point on a boundary), each
    traversed with the admitted cells on its left: the outer boundary runs
    counter-clockwise, the boundary around each excluded island clockwise.
    Raises if two loops touch at a vertex."""
    n = adm.shape[0]
    nxt = {}

    def a(i, j):
        return 0 <= i < n and 0 <= j < n and adm[i, j]

    def put(u, v):
        if u in nxt:
            raise RuntimeError("admitted cells touch at a corner only")
        nxt[u] = v

    for i, j in zip(*np.nonzero(adm)):
        i, j = int(i), int(j)
        if not a(i, j - 1):
            put((i, j), (i + 1, j))
        if not a(i + 1, j):
            put((i + 1, j), (i + 1, j + 1))
        if not a(i, j + 1):
            put((i + 1, j + 1), (i, j + 1))
        if not a(i - 1, j):
            put((i, j + 1), (i, j))
    loops, seen = [], set()
    for start in nxt:
        if start in seen:
            continue
        loop = [start]
        seen.add(start)
        v = nxt[start]
        while v != start:
            loop.append(v)
            seen.add(v)
            v = nxt[v]
        loops.append(np.array(loop))
    return loops


def _signed_area(poly):
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def _min_angle(a, b, c):
    out = []
    for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
        u, v = q - p, r - p
        out.append(math.acos(np.clip(np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v)), -1, 1)))
    return min(out)


def _orient(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1])


def _strip_band(stair, par, curve_pts, outward: bool):
    """Cut the gap between a closed staircase loop and a curve into strips, one
    per staircase edge, each bounded by the edge, the segments from its two
    vertices to their points on the curve, and the curve between those points;
    each strip is split into a curved triangle (first two vertices on the curve)
    and a straight one, along the diagonal with the larger minimum angle. A strip
    whose two curve points coincide is one straight triangle.
    stair [m, 2]: loop vertices ordered so that the curve parameter `par`
    (unwrapped, non-decreasing, total increase below 2 pi) increases;
    curve_pts [m, 2]: the curve at par. outward: the curve lies outside the
    staircase (outer boundary) or inside it (a hole).
    Returns [(kind, vertices[3, 2], (t0, t1) or None)]."""
    m = stair.shape[0]
    tris = []
    for j in range(m):
        j1 = (j + 1) % m
        th0 = par[j]
        th1 = par[j1] + (2 * math.pi if j1 == 0 else 0.0)
        Ij, Ij1, Oj, Oj1 = stair[j], stair[j1], curve_pts[j], curve_pts[j1]
        if th1 <= th0:
            tri = (Ij, Ij1, Oj) if outward else (Ij1, Ij, Oj)
            if _orient(*tri) <= 0:
                raise RuntimeError("inverted triangle in the band")
            tris.append((1, np.array(tri), None))
            continue
        if outward:   # counter-clockwise triangles: curve edge from th0 to th1
            splits = [((Oj, Oj1, Ij), (Ij, Ij1, Oj1), (th0, th1)),
                      ((Oj, Oj1, Ij1), (Oj, Ij1, Ij), (th0, th1))]
        else:         # curve inside: counter-clockwise means the curve edge runs from th1 to th0
            splits = [((Oj1, Oj, Ij), (Ij1, Ij, Oj1), (th1, th0)),
                      ((Oj1, Oj, Ij1), (Oj, Ij, Ij1), (th1, th0))]
        best = None
        for c_tri, s_tri, th in splits:
            if _orient(*c_tri) <= 0 or _orient(*s_tri) <= 0:
                continue
            q = min(_min_angle(*c_tri), _min_angle(*s_tri))
            if best is None or q > best[0]:
                best = (q, c_tri, s_tri, th)
        if best is None:
            raise RuntimeError("no valid split of a band strip")
        tris.append((2, np.array(best[1]), best[3]))
        tris.append((1, np.array(best[2]), None))
    return tris


def _radial_band(stair, centre, project, outward: bool):
    """Strips along rays from `centre` (the staircase must be strictly
    star-shaped about it); project(theta) -> point of the curve at polar angle
    theta about centre."""
    rel = stair - centre
    ang = np.arctan2(rel[:, 1], rel[:, 0])
    order = np.argsort(ang)
    stair, ang = stair[order], ang[order]
    if np.any(np.diff(ang) <= 0):
        raise RuntimeError("staircase is not strictly star-shaped about the centre")
    return _strip_band(stair, ang, np.array([project(t) for t in ang]), outward)


def _star_nearest(p, a: float, k: int, samples: int = 40000):
    """Polar angle of the point of the star boundary nearest to each row of p
    (dense sampling, then Newton on the squared distance)."""
    th = np.linspace(-math.pi, math.pi, samples, endpoint=False)
    r, _ = star_radius(th, a, k)
    from scipy.spatial import cKDTree

    _, idx = cKDTree(np.stack([r * np.cos(th), r * np.sin(th)], axis=1)).query(p)
    t = th[idx]
    for _ in range(8):
        r, dr = star_radius(t, a, k)
        ddr = -a * k * k * np.cos(k * t)
        c, s = np.cos(t), np.sin(t)
        x, y = r * c - p[:, 0], r * s - p[:, 1]
        xt, yt = dr * c - r * s, dr * s + r * c
        xtt, ytt = ddr * c - 2 * dr * s - r * c, ddr * s + 2 * dr * c - r * s
        g = x * xt + y * yt
        gp = xt * xt + yt * yt + x * xtt + y * ytt
        t = t - g / gp
    return t


def _normal_band_star(stair, a: float, k: int):
    """Strips from each vertex of the outer staircase (traversed counter-clockwise)
    to its nearest point on the star boundary; nearest-point parameters that step
    back along the loop are raised to their running maximum."""
    t = _star_nearest(stair, a, k)
    t0 = int(np.argmin(t))
    stair, t = np.roll(stair, -t0, axis=0), np.roll(t, -t0)
    t = np.unwrap(t)
    t = np.maximum.accumulate(t)
    if t[-1] - t[0] >= 2 * math.pi:
        raise RuntimeError("outer staircase winds more than once")
    r, _ = star_radius(t, a, k)
    return _strip_band(stair, t, np.stack([r * np.cos(t), r * np.sin(t)], axis=1), outward=True)


def _edge_samples(m: int = 12):
    """Points of the reference triangle on and near its edges, where a blended
    map folds first."""
    t = (np.arange(m) + 0.5) / m
    e = 1e-6
    xi = np.concatenate([t * (1 - e), np.full(m, e), (1 - t) * (1 - e)])
    eta = np.concatenate([np.full(m, e), t * (1 - e), t * (1 - e)])
    return xi, eta


def _box_point_dist(x0, y0, side, px, py):
    dx = np.maximum(np.maximum(x0 - px, 0.0), px - (x0 + side))
    dy = np.maximum(np.maximum(y0 - py, 0.0), py - (y0 + side))
    return np.hypot(dx, dy)


def star_holes(seed: int, count: int = 12, rmin: float = 0.02, rmax: float = 0.08, gap: float = 0.04,
               a: float = 0.3, k: int = 5):
    """`count` circular holes with radii uniform in [rmin, rmax], centres
    rejection-sampled inside the star so that hole-hole and hole-boundary gaps
    are at least `gap`. Returns [count, 3] (cx, cy, radius)."""
    rng = np.random.default_rng(seed)
    th = np.linspace(0, 2 * math.pi, 20000, endpoint=False)
    r, _ = star_radius(th, a, k)
    bnd = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    holes = []
    while len(holes) < count:
        rad = rng.uniform(rmin, rmax)
        p = rng.uniform(-1.3, 1.3, size=2)
        rp = math.hypot(p[0], p[1])
        if rp >= star_radius(math.atan2(p[1], p[0]), a, k)[0]:
            continue
        if np.min(np.hypot(bnd[:, 0] - p[0], bnd[:, 1] - p[1])) < rad + gap:
            continue
        if any(math.hypot(p[0] - hx, p[1] - hy) < rad + hr + gap for hx, hy, hr in holes):
            continue
        holes.append((float(p[0]), float(p[1]), float(rad)))
    return np.array(holes)


def inside_star(x, y, holes, a: float = 0.3, k: int = 5):
    """True where (x, y) lies inside the star and outside every hole."""
    r, _ = star_radius(np.arctan2(y, x), a, k)
    ok = np.hypot(x, y) < r
    for hx, hy, hr in holes:
        ok &= np.hypot(x - hx, y - hy) > hr
    return ok


def star_mesh(holes, base_level: int = 8, fine_level: int = 11, refine=None, delta: float = 0.8,
              box_order: int = 8, tri_p: int = 8, a: float = 0.3, k: int = 5, lo: float = -1.3,
              side: float = 2.6, tri_rule=None) -> Mesh:
    """Star r(theta) = 1 + a cos(k theta) with circular holes (rows cx, cy, R):
    uniform boxes of level `base_level` over [lo, lo + side]^2 kept where they
    lie inside the star at distance >= delta*h from its boundary and at distance
    >= R + delta*h from every hole centre; kept boxes are refined further by
    `refine(level, x0, y0, side) -> bool` up to `fine_level`. The gaps between
    the boxes' staircase boundaries and the curves are cut into radial strips
    about the origin (outer boundary) and about each hole centre, each strip
    split into a curved triangle (blending map of Eq. deformed_triangle_maps)
    and a straight one."""
    holes = np.asarray(holes, float).reshape(-1, 3)
    n = 1 << base_level
    h = side / n
    edges = lo + h * np.arange(n + 1)
    X0, Y0 = np.meshgrid(edges[:-1], edges[:-1], indexing="ij")
    # distance of each cell to the sampled boundary curve; spacing well below delta*h
    nth = int(2 * math.pi * 1.3 * 4 / h * 16)
    th = np.linspace(0, 2 * math.pi, nth, endpoint=False)
    rb, _ = star_radius(th, a, k)
    bnd = np.stack([rb * np.cos(th), rb * np.sin(th)], axis=1)
    spacing = float(np.max(np.hypot(*(np.roll(bnd, -1, axis=0) - bnd).T)))
    from scipy.spatial import cKDTree

    tree = cKDTree(bnd)
    cx, cy = X0 + h / 2, Y0 + h / 2
    inside = inside_star(cx.ravel(), cy.ravel(), np.zeros((0, 3)), a, k).reshape(n, n)
    near = tree.query_ball_point(np.stack([cx.ravel(), cy.ravel()], axis=1), r=h / math.sqrt(2) + delta * h + spacing)
    adm = inside.copy()
    for idx, lst in enumerate(near):
        if not adm.flat[idx] or not lst:
            continue
        i, j = divmod(idx, n)
        pts = bnd[lst]
        if np.min(_box_point_dist(X0[i, j], Y0[i, j], h, pts[:, 0], pts[:, 1])) < delta * h + spacing:
            adm[i, j] = False
    for hx, hy, hr in holes:
        adm &= _box_point_dist(X0, Y0, h, hx, hy) >= hr + delta * h
    # two kept cells that share only a corner pinch the boundary: drop one of them
    while True:
        a00, a10, a01, a11 = adm[:-1, :-1], adm[1:, :-1], adm[:-1, 1:], adm[1:, 1:]
        pinch = (a00 & a11 & ~a10 & ~a01) | (a10 & a01 & ~a00 & ~a11)
        if not pinch.any():
            break
        for i, j in zip(*np.nonzero(pinch)):
            cand = [(i, j), (i + 1, j + 1)] if adm[i, j] and adm[i + 1, j + 1] else [(i + 1, j), (i, j + 1)]
            drop = max(cand, key=lambda c: math.hypot(cx[c], cy[c]))
            adm[drop] = False

    boxes = []
    stack = [(base_level, float(X0[i, j]), float(Y0[i, j]), h) for i, j in zip(*np.nonzero(adm))]
    while stack:
        lvl, x0, y0, s = stack.pop()
        if refine is not None and lvl < fine_level and refine(lvl, x0, y0, s):
            s2 = s / 2
            stack.extend([(lvl + 1, x0, y0, s2), (lvl + 1, x0 + s2, y0, s2), (lvl + 1, x0, y0 + s2, s2),
                          (lvl + 1, x0 + s2, y0 + s2, s2)])
        else:
            boxes.append((lvl, x0, y0, s))
    boxes.sort(key=lambda b: (b[0], b[2], b[1]))

    loops = [lp.astype(float) * h + lo for lp in _staircase_loops(adm)]
    outer = [lp for lp in loops if _signed_area(lp) > 0]
    inner = [lp for lp in loops if _signed_area(lp) < 0]
    if len(outer) != 1 or len(inner) != holes.shape[0]:
        raise RuntimeError(f"expected one outer boundary and {holes.shape[0]} hole boundaries, "
                           f"got {len(outer)} and {len(inner)}")
    tris = _normal_band_star(outer[0], a, k)
    arcs = [None] * len(tris)
    for t in range(len(tris)):
        if tris[t][0] == 2:
            arcs[t] = ("star", None)
    for hx, hy, hr in holes:
        c = np.array([hx, hy])
        mine = [lp for lp in inner if np.all(np.hypot(lp[:, 0] - hx, lp[:, 1] - hy) > hr)
                and np.max(np.hypot(lp[:, 0] - hx, lp[:, 1] - hy)) < hr + 4 * h]
        if len(mine) != 1:
            raise RuntimeError("could not match a hole to its staircase boundary")
        ht = _radial_band(mine[0], c, lambda t, c=c, hr=hr: c + hr * np.array([math.cos(t), math.sin(t)]),
                          outward=False)
        tris.extend(ht)
        arcs.extend([("circle", (hx, hy, hr)) if tk == 2 else None for tk, _, _ in ht])

    txi, teta, tw = simplex.simplex_rule(tri_p) if tri_rule is None else tri_rule
    bx, by, bw = simplex.gauss_legendre_box(box_order)
    xs, ws, start, bbox, kind, level = [], [], [0], [], [], []
    geom = []
    for (tk, v, thr), arc in zip(tris, arcs):
        curve = None
        if tk == 2:
            if arc[0] == "star":
                curve = star_curve(thr[0], thr[1], a, k)
            else:
                curve = simplex.circle_arc(arc[1][0], arc[1][1], arc[1][2], thr[0], thr[1])
        geom.append(("tri", v, curve))
        if tk == 2:
            pts, J = simplex.blended_map(v, curve, txi, teta, signed=True)
            # the map must not fold: det DR keeps the sign of the counter-clockwise vertices
            if np.any(J <= 0) or np.any(simplex.blended_map(v, curve, *_edge_samples(), signed=True)[1] <= 0):
                raise RuntimeError("folded curved triangle in the band")
            sx, sy, _, _ = curve(np.linspace(0, 1, 9))
            bb = [min(v[:, 0].min(), sx.min()), max(v[:, 0].max(), sx.max()),
                  min(v[:, 1].min(), sy.min()), max(v[:, 1].max(), sy.max())]
        else:
            pts, J = simplex.affine_map(v, txi, teta)
            bb = [v[:, 0].min(), v[:, 0].max(), v[:, 1].min(), v[:, 1].max()]
        if np.any(J <= 0):
            raise RuntimeError("degenerate triangle in the band")
        xs.append(pts)
        ws.append(tw * J)
        start.append(start[-1] + pts.shape[0])
        bbox.append(bb)
        kind.append(tk)
        level.append(-1)
    for lvl, x0, y0, s in boxes:
        half = s / 2
        xs.append(np.stack([x0 + half + half * bx, y0 + half + half * by], axis=1))
        ws.append(bw * half * half)
        start.append(start[-1] + bx.size)
        bbox.append([x0, x0 + s, y0, y0 + s])
        kind.append(0)
        level.append(lvl)
        geom.append(("box", x0, y0, s))
    area = math.pi * (1.0 + a * a / 2.0) - float(np.sum(math.pi * holes[:, 2] ** 2))
    return Mesh(xy=np.ascontiguousarray(np.vstack(xs)), w=np.concatenate(ws),
                cell_start=np.array(start, np.int64), cell_bbox=np.array(bbox), cell_kind=np.array(kind, np.int8),
                cell_level=np.array(level, np.int32), area=area, geom=geom)
