"""SIPG assembly (Sec. 2, Eq. dG, Eq. Ah, Eq. lifting, Eq. Sigma).

The lifted form of Eq. Ah equals the weighted interior-penalty form: rho grad_h u lies in [V_h]^2
because rho is constant per element (Remark 2.1), so it is an admissible eta in the lifting
definition and int rho grad_h u . R_rho([[v]]) = - int_F [[v]] . {rho grad_h u}_omega.  With
omega = rho^- / (rho^+ + rho^-) on interior faces, {rho grad u}_omega = <rho>/2 (grad u^+ + grad u^-)
where <rho> = 2 rho^+ rho^- / (rho^+ + rho^-) is the harmonic average; on boundary faces
{rho grad u}_omega = rho_kappa grad u and [[v]] = v n.

For test function phi_a on side s_a and trial function phi_b on side s_b of an interior face
(s = +1 on kappa^+, -1 on kappa^-, n = n_{kappa^+}) the face contributes
    A[a, b] += int_F ( -<rho>/2 s_a phi_a d_n phi_b - <rho>/2 s_b phi_b d_n phi_a
                       + sigma s_a s_b phi_a phi_b ),
sigma = C_sigma <rho> p^2 / <h_kappa> (Eq. Sigma), and a boundary face of kappa contributes
    A[a, b] += int_F ( -rho phi_a d_n phi_b - rho phi_b d_n phi_a + sigma phi_a phi_b ),
sigma = C_sigma rho_kappa p^2 / h_kappa.  Elements contribute rho_kappa int grad phi_a . grad phi_b.
The load vector is b_a = int f phi_a (zero Dirichlet data).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import eval_basis, n_basis
from .geometry import build_geometry
from .quadrature import polygon_rule, segment_rule


def harmonic(a: float, b: float) -> float:
    return 2.0 * a * b / (a + b)


def assemble(mesh, rho, p: int, c_sigma: float = 10.0, f=None, geom=None):
    """Returns (A as scipy CSR, b or None, geometry).  Dof of basis a on element e is e * n_p + a."""
    geom = build_geometry(mesh) if geom is None else geom
    rho = np.asarray(rho, dtype=np.float64)
    nb = n_basis(p)
    ne = mesh.n_elem
    rows, cols, vals = [], [], []

    def add_block(ea, eb, blk):
        ia = ea * nb + np.arange(nb)
        ib = eb * nb + np.arange(nb)
        rows.append(np.repeat(ia, nb))
        cols.append(np.tile(ib, nb))
        vals.append(blk.ravel())

    m_mat = p + 2
    b = np.zeros(ne * nb) if f is not None else None
    for e in range(ne):
        poly = mesh.polygon(e)
        pts, w = polygon_rule(poly, m_mat)
        _, grad = eval_basis(p, geom.bbox[e], pts)
        # K[a, b] = rho int grad phi_a . grad phi_b
        K = rho[e] * np.einsum("q,qad,qbd->ab", w, grad, grad)
        add_block(e, e, K)
        if f is not None:
            pts_f, w_f = polygon_rule(poly, p + 5)
            val_f, _ = eval_basis(p, geom.bbox[e], pts_f)
            b[e * nb:(e + 1) * nb] = val_f.T @ (w_f * f(pts_f))

    for (ep, em, va, vb) in geom.faces:
        xa, xb = mesh.xy[va], mesh.xy[vb]
        pts, w = segment_rule(xa, xb, m_mat)
        d = xb - xa
        n = np.array([d[1], -d[0]]) / np.hypot(d[0], d[1])
        if em < 0:
            sigma = c_sigma * rho[ep] * p * p / geom.diameter[ep]
            v, g = eval_basis(p, geom.bbox[ep], pts)
            dn = g @ n
            blk = (np.einsum("q,qa,qb->ab", w, v, -rho[ep] * dn)
                   + np.einsum("q,qb,qa->ab", w, v, -rho[ep] * dn)
                   + sigma * np.einsum("q,qa,qb->ab", w, v, v))
            add_block(ep, ep, blk)
            continue
        rho_avg = harmonic(rho[ep], rho[em])
        h_avg = harmonic(geom.diameter[ep], geom.diameter[em])
        sigma = c_sigma * rho_avg * p * p / h_avg
        side = {}
        for e, s in ((ep, 1.0), (em, -1.0)):
            v, g = eval_basis(p, geom.bbox[e], pts)
            side[e] = (s, v, g @ n)
        for ea in (ep, em):
            sa, va_, dna = side[ea]
            for eb in (ep, em):
                sb, vb_, dnb = side[eb]
                blk = (-0.5 * rho_avg * sa * np.einsum("q,qa,qb->ab", w, va_, dnb)
                       - 0.5 * rho_avg * sb * np.einsum("q,qb,qa->ab", w, vb_, dna)
                       + sigma * sa * sb * np.einsum("q,qa,qb->ab", w, va_, vb_))
                add_block(ea, eb, blk)

    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ne * nb, ne * nb)).tocsr()
    A.sum_duplicates()
    return A, b, geom


def mass_blocks(mesh, p: int, geom):
    """Element mass matrices M_kappa[a, b] = int_kappa phi_a phi_b."""
    out = []
    for e in range(mesh.n_elem):
        pts, w = polygon_rule(mesh.polygon(e), p + 2)
        v, _ = eval_basis(p, geom.bbox[e], pts)
        out.append(np.einsum("q,qa,qb->ab", w, v, v))
    return out
