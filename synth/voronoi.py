"""Lloyd-relaxed Voronoi tessellations of the unit square.

Seeds are drawn uniformly in (0,1)^2 from ``numpy.random.default_rng(seed)``.  Each Lloyd step
replaces every seed by the area centroid of its cell.  Cells are clipped to the square by adding
the mirror images of all seeds across the four sides: the bisector between a seed and its mirror
is the side itself, and a mirrored seed is never closer to a point of the square than its
original, so the cell of an original seed in the augmented diagram equals its Voronoi cell
intersected with the square.

Vertices closer than ``weld_tol`` are merged (degenerate four-cell junctions, e.g. at the
corners, come out of qhull as two nearly coincident vertices), coordinates within ``weld_tol``
of a side are snapped onto it, and repeated consecutive vertices are dropped.  Polygons are
returned counter-clockwise.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.spatial import Voronoi, cKDTree


@dataclass
class PolyMesh:
    """A polygonal mesh: vertex coordinates and a CSR list of CCW polygon vertex ids."""
    xy: np.ndarray        # (nv, 2) float64
    poly_ptr: np.ndarray  # (ne + 1,) int32
    poly_vtx: np.ndarray  # (poly_ptr[-1],) int32

    @property
    def n_elem(self) -> int:
        return len(self.poly_ptr) - 1

    def polygon(self, e: int) -> np.ndarray:
        return self.xy[self.poly_vtx[self.poly_ptr[e]:self.poly_ptr[e + 1]]]


def polygon_area_centroid(xy: np.ndarray, poly_ptr: np.ndarray, poly_vtx: np.ndarray):
    """Signed areas and area centroids of all polygons (shoelace formula), vectorised."""
    ne = len(poly_ptr) - 1
    counts = np.diff(poly_ptr)
    start = np.repeat(poly_ptr[:-1], counts)
    local = np.arange(len(poly_vtx)) - start
    nxt = start + (local + 1) % np.repeat(counts, counts)
    p0 = xy[poly_vtx]
    p1 = xy[poly_vtx[nxt]]
    cross = p0[:, 0] * p1[:, 1] - p1[:, 0] * p0[:, 1]
    seg = np.repeat(np.arange(ne), counts)
    a2 = np.bincount(seg, weights=cross, minlength=ne)
    cx = np.bincount(seg, weights=(p0[:, 0] + p1[:, 0]) * cross, minlength=ne)
    cy = np.bincount(seg, weights=(p0[:, 1] + p1[:, 1]) * cross, minlength=ne)
    area = 0.5 * a2
    cen = np.stack([cx / (3.0 * a2), cy / (3.0 * a2)], axis=1)
    return area, cen


def _clipped_cells(pts: np.ndarray):
    n = len(pts)
    # Mirror the seeds within ``band`` of a side; widen the band until every original cell is
    # bounded and lies inside the square (a far-away seed's mirror can never bound a cell).
    band = min(1.0, 4.0 / np.sqrt(n))
    while True:
        x, y = pts[:, 0], pts[:, 1]
        parts = [pts]
        for sel, img in ((x < band, np.stack([-x, y], 1)), (x > 1.0 - band, np.stack([2.0 - x, y], 1)),
                         (y < band, np.stack([x, -y], 1)), (y > 1.0 - band, np.stack([x, 2.0 - y], 1))):
            parts.append(img[sel])
        aug = np.concatenate(parts)
        vor = Voronoi(aug)
        regions = [vor.regions[vor.point_region[i]] for i in range(n)]
        ok = all(len(r) >= 3 and -1 not in r for r in regions)
        if ok:
            counts = np.array([len(r) for r in regions], dtype=np.int64)
            ptr = np.zeros(n + 1, dtype=np.int64)
            np.cumsum(counts, out=ptr[1:])
            vtx = np.fromiter((v for r in regions for v in r), dtype=np.int64, count=int(ptr[-1]))
            v = vor.vertices[vtx]
            if v.min() > -1e-9 and v.max() < 1.0 + 1e-9:
                return vor.vertices.copy(), ptr, vtx
        if band >= 1.0:
            raise RuntimeError("could not clip the Voronoi diagram to the unit square")
        band = min(1.0, 2.0 * band)


def _orient_ccw(xy, ptr, vtx):
    area, _ = polygon_area_centroid(xy, ptr, vtx)
    vtx = vtx.copy()
    for e in np.nonzero(area < 0)[0]:
        vtx[ptr[e]:ptr[e + 1]] = vtx[ptr[e]:ptr[e + 1]][::-1]
    return vtx


def _weld(xy, ptr, vtx, tol):
    used = np.unique(vtx)
    pos = xy[used].copy()
    for d in range(2):
        c = pos[:, d]
        c[np.abs(c) < tol] = 0.0
        c[np.abs(c - 1.0) < tol] = 1.0
        np.clip(c, 0.0, 1.0, out=c)
    # union-find over vertex pairs closer than tol
    parent = np.arange(len(used))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in sorted(cKDTree(pos).query_pairs(r=tol)):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(a) for a in range(len(used))])
    uniq_roots, new_id = np.unique(roots, return_inverse=True)
    new_xy = pos[uniq_roots]
    remap = np.full(xy.shape[0], -1, dtype=np.int64)
    remap[used] = new_id
    nv = remap[vtx]
    out_ptr = [0]
    out_vtx = []
    for e in range(len(ptr) - 1):
        ring = list(nv[ptr[e]:ptr[e + 1]])
        cleaned = []
        for v in ring:
            if not cleaned or cleaned[-1] != v:
                cleaned.append(v)
        while len(cleaned) > 1 and cleaned[0] == cleaned[-1]:
            cleaned.pop()
        if len(cleaned) < 3:
            raise RuntimeError(f"polygon {e} collapsed while welding")
        out_vtx.extend(cleaned)
        out_ptr.append(len(out_vtx))
    return new_xy, np.asarray(out_ptr, dtype=np.int32), np.asarray(out_vtx, dtype=np.int32)


def voronoi_mesh(n: int, seed: int, lloyd: int = 20, weld_tol: float = 1e-12) -> PolyMesh:
    """Clipped, Lloyd-relaxed Voronoi mesh of (0,1)^2 with ``n`` cells."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    for _ in range(lloyd):
        xy, ptr, vtx = _clipped_cells(pts)
        vtx = _orient_ccw(xy, ptr, vtx)
        _, cen = polygon_area_centroid(xy, ptr, vtx)
        pts = cen
    xy, ptr, vtx = _clipped_cells(pts)
    vtx = _orient_ccw(xy, ptr, vtx)
    xy, ptr, vtx = _weld(xy, ptr, vtx, weld_tol)
    return PolyMesh(xy=np.ascontiguousarray(xy, dtype=np.float64), poly_ptr=ptr, poly_vtx=vtx)


def quad_mesh(nx: int, ny: int | None = None) -> PolyMesh:
    """Structured nx-by-ny mesh of unit-square cells (squares as 4-gons), row-major element order."""
    ny = nx if ny is None else ny
    xs = np.linspace(0.0, 1.0, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    vid = lambda i, j: j * (nx + 1) + i  # noqa: E731
    vtx = []
    for j in range(ny):
        for i in range(nx):
            vtx += [vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)]
    ptr = np.arange(0, 4 * nx * ny + 1, 4, dtype=np.int32)
    return PolyMesh(xy=xy, poly_ptr=ptr, poly_vtx=np.asarray(vtx, dtype=np.int32))
