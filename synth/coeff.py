"""Piecewise-constant diffusion coefficients and random right-hand sides (inputs only)."""
from __future__ import annotations

import numpy as np

from .voronoi import PolyMesh, polygon_area_centroid


def _sub_centroids(mesh: PolyMesh, sub_of_elem: np.ndarray):
    area, cen = polygon_area_centroid(mesh.xy, mesh.poly_ptr, mesh.poly_vtx)
    ns = int(sub_of_elem.max()) + 1
    w = np.bincount(sub_of_elem, weights=area, minlength=ns)
    cx = np.bincount(sub_of_elem, weights=area * cen[:, 0], minlength=ns) / w
    cy = np.bincount(sub_of_elem, weights=area * cen[:, 1], minlength=ns) / w
    return cx, cy


def checker_per_subdomain(mesh: PolyMesh, sub_of_elem: np.ndarray, contrast: float,
                          cells: int = 4) -> np.ndarray:
    """rho = contrast on subdomains whose area centroid lies in an odd cell of a cells x cells
    checkerboard of the unit square, 1 elsewhere; constant on every subdomain."""
    cx, cy = _sub_centroids(mesh, sub_of_elem)
    odd = (np.floor(cells * cx).astype(int) + np.floor(cells * cy).astype(int)) % 2 == 1
    rho_sub = np.where(odd, float(contrast), 1.0)
    return rho_sub[sub_of_elem].astype(np.float64)


def checker_per_element(mesh: PolyMesh, contrast: float, cells: int = 4) -> np.ndarray:
    """Checkerboard evaluated at each element's area centroid (not aligned with subdomains)."""
    _, cen = polygon_area_centroid(mesh.xy, mesh.poly_ptr, mesh.poly_vtx)
    odd = (np.floor(cells * cen[:, 0]).astype(int) + np.floor(cells * cen[:, 1]).astype(int)) % 2 == 1
    return np.where(odd, float(contrast), 1.0).astype(np.float64)


def loguniform_per_subdomain(sub_of_elem: np.ndarray, rng: np.random.Generator,
                             lo: float = 1.0, hi: float = 1e3) -> np.ndarray:
    """rho = 10**U(log10 lo, log10 hi), one draw per subdomain."""
    ns = int(sub_of_elem.max()) + 1
    rho_sub = 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), size=ns)
    return rho_sub[sub_of_elem].astype(np.float64)
