"""L2 error of a DG solution against an exact solution, by element quadrature (m = p + 5)."""
from __future__ import annotations

import numpy as np

from .basis import eval_basis, n_basis
from .quadrature import polygon_rule


def l2_error(mesh, geom, p: int, x: np.ndarray, u_exact) -> float:
    nb = n_basis(p)
    total = 0.0
    for e in range(mesh.n_elem):
        pts, w = polygon_rule(mesh.polygon(e), p + 5)
        v, _ = eval_basis(p, geom.bbox[e], pts)
        uh = v @ x[e * nb:(e + 1) * nb]
        total += float(w @ (uh - u_exact(pts)) ** 2)
    return float(np.sqrt(total))


def l2_projection(mesh, geom, p: int, u):
    """Coefficients of the elementwise L2 projection of u onto V_h."""
    nb = n_basis(p)
    out = np.empty(mesh.n_elem * nb)
    for e in range(mesh.n_elem):
        pts, w = polygon_rule(mesh.polygon(e), p + 5)
        v, _ = eval_basis(p, geom.bbox[e], pts)
        M = np.einsum("q,qa,qb->ab", w, v, v)
        out[e * nb:(e + 1) * nb] = np.linalg.solve(M, v.T @ (w * u(pts)))
    return out
