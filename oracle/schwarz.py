"""Two-level non-overlapping additive Schwarz preconditioner (Sec. 3).

Local solvers: V_i = V_h restricted to Omega_i, A_i(u, v) = A_h(R_i^T u, R_i^T v) with R_i^T the
extension by zero, so the matrix of A_i is the principal submatrix of A on the dofs of Omega_i.
Coarse solver: V_0 = polynomials of degree q on each agglomerate D_j (basis: scaled Legendre
products on D_j's bounding box, as for the fine space), R_0^T the L2 prolongation of Eq. R0T
(per element kappa in D_j, R_0^T|_kappa = M_kappa^{-1} N_kappa with M_kappa = int phi phi^T and
N_kappa = int phi psi_j^T), and A_0 = R_0 A R_0^T (Eq. A0) with R_0 = (R_0^T)^T.  The coarse elements D_j
may instead be the cells of an independent (non-nested) polygonal mesh, as in Example 4: then kappa meets
several D_j and R_0^T|_kappa = M_kappa^{-1} [int_{kappa cap D_j} phi psi_j^T]_j.

From the definitions of P_i and P_0 (Sec. 3), P_ad = B A with
    B = R_0^T A_0^{-1} R_0 + sum_i R_i^T A_i^{-1} R_i,
so applying the preconditioner to a residual r is z = B r.  Local and coarse systems are solved
with dense Cholesky factors (numpy / scipy).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .basis import eval_basis, n_basis
from .quadrature import polygon_rule


@dataclass
class Schwarz:
    local_dofs: list        # [np.ndarray] dofs of each subdomain (ascending)
    local_chol: list        # [np.ndarray] lower Cholesky factors of A_i
    R0T: sp.csr_matrix      # (ndof, n0) prolongation, or None
    A0: np.ndarray          # (n0, n0) or None
    A0_chol: np.ndarray     # lower Cholesky factor of A0 or None

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros_like(r)
        for idx, L in zip(self.local_dofs, self.local_chol):
            y = sla.solve_triangular(L, r[idx], lower=True)
            z[idx] += sla.solve_triangular(L, y, lower=True, trans="T")
        if self.R0T is not None:
            r0 = self.R0T.T @ r
            y0 = sla.solve_triangular(self.A0_chol, r0, lower=True)
            z0 = sla.solve_triangular(self.A0_chol, y0, lower=True, trans="T")
            z += self.R0T @ z0
        return z

    def dense(self, ndof: int) -> np.ndarray:
        """B as a dense matrix (tiny meshes only)."""
        return np.stack([self.apply(col) for col in np.eye(ndof)], axis=1)


def local_dof_sets(sub: np.ndarray, nb: int) -> list:
    ns = int(sub.max()) + 1
    out = []
    for i in range(ns):
        elems = np.nonzero(sub == i)[0]
        out.append((elems[:, None] * nb + np.arange(nb)[None, :]).ravel())
    return out


def agglomerate_boxes(mesh, agg: np.ndarray, geom) -> np.ndarray:
    nagg = int(agg.max()) + 1
    box = np.empty((nagg, 4))
    box[:, 0] = np.inf
    box[:, 1] = -np.inf
    box[:, 2] = np.inf
    box[:, 3] = -np.inf
    for e in range(mesh.n_elem):
        j = agg[e]
        b = geom.bbox[e]
        box[j] = (min(box[j, 0], b[0]), max(box[j, 1], b[1]), min(box[j, 2], b[2]), max(box[j, 3], b[3]))
    return box


def prolongation(mesh, geom, agg: np.ndarray, p: int, q: int) -> sp.csr_matrix:
    """R_0^T of Eq. R0T for nested agglomerates: block M_kappa^{-1} N_kappa per element."""
    nb = n_basis(p)
    nq = n_basis(q)
    boxes = agglomerate_boxes(mesh, agg, geom)
    nagg = len(boxes)
    rows, cols, vals = [], [], []
    for e in range(mesh.n_elem):
        pts, w = polygon_rule(mesh.polygon(e), p + 2)
        phi, _ = eval_basis(p, geom.bbox[e], pts)
        psi, _ = eval_basis(q, boxes[agg[e]], pts)
        M = np.einsum("q,qa,qb->ab", w, phi, phi)
        N = np.einsum("q,qa,qc->ac", w, phi, psi)
        blk = np.linalg.solve(M, N)
        r = e * nb + np.arange(nb)
        c = agg[e] * nq + np.arange(nq)
        rows.append(np.repeat(r, nq))
        cols.append(np.tile(c, nb))
        vals.append(blk.ravel())
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(mesh.n_elem * nb, nagg * nq)).tocsr()


def clip_convex(subject: np.ndarray, clip: np.ndarray) -> np.ndarray:
    """Part of polygon `subject` inside the convex counter-clockwise polygon `clip` (Sutherland-Hodgman:
    clip against the half-plane left of each edge of `clip` in turn).  Returns the vertices (k, 2), k may
    be 0."""
    out = [np.asarray(v, dtype=np.float64) for v in subject]
    n = len(clip)
    for i in range(n):
        a = np.asarray(clip[i], dtype=np.float64)
        b = np.asarray(clip[(i + 1) % n], dtype=np.float64)
        if not out:
            break
        inp = out
        out = []

        def side(v):
            return (b[0] - a[0]) * (v[1] - a[1]) - (b[1] - a[1]) * (v[0] - a[0])

        for k in range(len(inp)):
            cur = inp[k]
            prev = inp[k - 1]
            sc, sp_ = side(cur), side(prev)
            if sc >= 0.0:
                if sp_ < 0.0:
                    out.append(prev + (cur - prev) * (sp_ / (sp_ - sc)))
                out.append(cur)
            elif sp_ >= 0.0:
                out.append(prev + (cur - prev) * (sp_ / (sp_ - sc)))
    return np.array(out).reshape(-1, 2)


def polygon_area(poly: np.ndarray) -> float:
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * float(np.dot(x, np.roll(y, -1)) - np.dot(np.roll(x, -1), y))


def prolongation_nonnested(mesh, geom, cmesh, cgeom, p: int, q: int, min_rel_area: float = 1e-12) -> sp.csr_matrix:
    """R_0^T of Eq. R0T for a coarse mesh that is not an agglomeration of the fine one (Example 4): on each
    fine element kappa, R_0^T v_0 is the L2 projection of the piecewise polynomial v_0, so
    R_0^T|_kappa = M_kappa^{-1} [N_kappa,j]_j with N_kappa,j = int_{kappa cap D_j} phi psi_j^T over every coarse
    element D_j that overlaps kappa (pieces by convex clipping, integrated with the element rule).  Pieces
    below min_rel_area |kappa| are dropped."""
    nb = n_basis(p)
    nq = n_basis(q)
    nc = cmesh.n_elem
    cb = cgeom.bbox
    rows, cols, vals = [], [], []
    for e in range(mesh.n_elem):
        poly = mesh.polygon(e)
        pts, w = polygon_rule(poly, p + 2)
        phi, _ = eval_basis(p, geom.bbox[e], pts)
        M = np.einsum("q,qa,qb->ab", w, phi, phi)
        b = geom.bbox[e]
        cand = np.nonzero((cb[:, 0] < b[1]) & (cb[:, 1] > b[0]) & (cb[:, 2] < b[3]) & (cb[:, 3] > b[2]))[0]
        area_e = polygon_area(poly)
        for j in cand:
            piece = clip_convex(poly, cmesh.polygon(j))
            if len(piece) < 3 or polygon_area(piece) <= min_rel_area * area_e:
                continue
            pp, pw = polygon_rule(piece, p + 2)
            ph, _ = eval_basis(p, geom.bbox[e], pp)
            ps, _ = eval_basis(q, cb[j], pp)
            blk = np.linalg.solve(M, np.einsum("q,qa,qc->ac", pw, ph, ps))
            r = e * nb + np.arange(nb)
            c = j * nq + np.arange(nq)
            rows.append(np.repeat(r, nq))
            cols.append(np.tile(c, nb))
            vals.append(blk.ravel())
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(mesh.n_elem * nb, nc * nq)).tocsr()


def build(A: sp.spmatrix, mesh, geom, p: int, sub: np.ndarray, agg=None, q: int = 1, coarse=None) -> Schwarz:
    """coarse: optional (coarse mesh, its geometry) of a non-nested coarse space; agg is then ignored."""
    nb = n_basis(p)
    A = sp.csr_matrix(A)
    dofs = local_dof_sets(sub, nb)
    chol = []
    for idx in dofs:
        Ai = A[idx][:, idx].toarray()
        chol.append(np.linalg.cholesky(Ai))
    R0T = A0 = L0 = None
    if coarse is not None:
        R0T = prolongation_nonnested(mesh, geom, coarse[0], coarse[1], p, q)
    elif agg is not None:
        R0T = prolongation(mesh, geom, agg, p, q)
    if R0T is not None:
        A0 = (R0T.T @ (A @ R0T)).toarray()
        A0 = 0.5 * (A0 + A0.T)
        L0 = np.linalg.cholesky(A0)
    return Schwarz(local_dofs=dofs, local_chol=chol, R0T=R0T, A0=A0, A0_chol=L0)
