"""Mesh geometry and faces (Sec. 2: elements kappa of diameter h_kappa, faces F_h = F_h^I u F_h^B).

Faces are the edges of the CCW polygons.  An edge (a, b) of one polygon whose reverse (b, a) is an
edge of another polygon is an interior face; otherwise it is a boundary face.  Interior faces are
stored with kappa^+ = the lower element index and the vertex pair in kappa^+'s CCW order, so the
outward unit normal of kappa^+ is (dy, -dx) / |F|.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Geometry:
    area: np.ndarray       # (ne,)
    centroid: np.ndarray   # (ne, 2) area centroid
    diameter: np.ndarray   # (ne,) h_kappa = max vertex-pair distance
    bbox: np.ndarray       # (ne, 4) x0, x1, y0, y1
    faces: list            # [(e_plus, e_minus or -1, va, vb)]


def polygon_area_centroid_loop(poly: np.ndarray):
    """Shoelace area and area centroid, summed vertex by vertex from vertex 0."""
    n = len(poly)
    a2 = 0.0
    cx = 0.0
    cy = 0.0
    for k in range(n):
        x0, y0 = poly[k]
        x1, y1 = poly[(k + 1) % n]
        cr = x0 * y1 - x1 * y0
        a2 += cr
        cx += (x0 + x1) * cr
        cy += (y0 + y1) * cr
    return 0.5 * a2, (cx / (3.0 * a2), cy / (3.0 * a2))


def diameter(poly: np.ndarray) -> float:
    best = 0.0
    for i in range(len(poly)):
        for j in range(i + 1, len(poly)):
            best = max(best, math.hypot(poly[i, 0] - poly[j, 0], poly[i, 1] - poly[j, 1]))
    return best


def build_geometry(mesh) -> Geometry:
    ne = mesh.n_elem
    area = np.empty(ne)
    cen = np.empty((ne, 2))
    diam = np.empty(ne)
    bbox = np.empty((ne, 4))
    edges = {}
    for e in range(ne):
        ids = mesh.poly_vtx[mesh.poly_ptr[e]:mesh.poly_ptr[e + 1]]
        poly = mesh.xy[ids]
        area[e], cen[e] = polygon_area_centroid_loop(poly)
        diam[e] = diameter(poly)
        bbox[e] = (poly[:, 0].min(), poly[:, 0].max(), poly[:, 1].min(), poly[:, 1].max())
        for k in range(len(ids)):
            edges[(int(ids[k]), int(ids[(k + 1) % len(ids)]))] = e
    faces = []
    for (a, b), e in edges.items():
        other = edges.get((b, a))
        if other is None:
            faces.append((e, -1, a, b))
        elif e < other:
            faces.append((e, other, a, b))
    faces.sort()
    return Geometry(area=area, centroid=cen, diameter=diam, bbox=bbox, faces=faces)
