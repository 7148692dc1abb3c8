"""Seeded synthetic inputs: clipped Voronoi meshes, coefficient patterns and right-hand sides.

This module holds no arithmetic of the solver method (no SIPG, no Schwarz preconditioner,
no Krylov iteration).  It only produces inputs: polygon meshes of the unit square, piecewise
constant diffusion coefficients and random vectors.  Both the library and the CPU oracle
consume these inputs.
"""
from .voronoi import PolyMesh, voronoi_mesh, polygon_area_centroid
from .coeff import checker_per_subdomain, loguniform_per_subdomain, checker_per_element

__all__ = ["PolyMesh", "voronoi_mesh", "polygon_area_centroid", "checker_per_subdomain",
           "loguniform_per_subdomain", "checker_per_element"]
