"""Pins of the oracle's non-nested coarse space (Eq. R0T with an independent coarse mesh, Example 4).

R_0^T v_0 is the L2 projection of the coarse function onto V_h, computed piece by piece over the
intersections of fine and coarse cells.  What the mathematics fixes, independently of that code:
  * the pieces of a fine cell tile it, and the pieces of a coarse cell tile it (areas add up);
  * a global polynomial of degree <= q lies in V_0 and in V_h, so R_0^T reproduces it exactly;
  * with the coarse mesh equal to the fine mesh, R_0^T is the nested injection (Remark 3.1), which the
    nested code computes by another route (one agglomerate per element, no clipping);
  * the Schwarz operator built on it is symmetric positive definite and PCG with it reaches the solution.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import partition, pcg, schwarz, sipg
from oracle.basis import eval_basis, n_basis
from oracle.geometry import build_geometry
from oracle.quadrature import polygon_rule
from tests.helpers import f_sin, mesh


def _pair(nf, nc, seed_f=3, seed_c=11):
    fm, cm = mesh(nf, seed_f), mesh(nc, seed_c)
    return fm, build_geometry(fm), cm, build_geometry(cm)


def test_clip_convex_square_cases():
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    shifted = sq + [0.5, 0.25]
    piece = schwarz.clip_convex(shifted, sq)
    assert abs(schwarz.polygon_area(piece) - 0.5 * 0.75) < 1e-15
    assert len(schwarz.clip_convex(sq + [2.0, 0.0], sq)) == 0          # disjoint
    inner = 0.25 + 0.5 * sq
    assert abs(schwarz.polygon_area(schwarz.clip_convex(inner, sq)) - 0.25) < 1e-15   # contained
    tri = np.array([[-1, -1], [3, -1], [-1, 3]], float)                # square inside a triangle
    assert abs(schwarz.polygon_area(schwarz.clip_convex(sq, tri)) - 1.0) < 1e-15


def test_pieces_tile_fine_and_coarse_cells():
    fm, fg, cm, cg = _pair(120, 17)
    fine_sum = np.zeros(fm.n_elem)
    coarse_sum = np.zeros(cm.n_elem)
    for e in range(fm.n_elem):
        for j in range(cm.n_elem):
            piece = schwarz.clip_convex(fm.polygon(e), cm.polygon(j))
            if len(piece) >= 3:
                a = schwarz.polygon_area(piece)
                fine_sum[e] += a
                coarse_sum[j] += a
    fa = np.array([schwarz.polygon_area(fm.polygon(e)) for e in range(fm.n_elem)])
    ca = np.array([schwarz.polygon_area(cm.polygon(j)) for j in range(cm.n_elem)])
    assert np.allclose(fine_sum, fa, rtol=1e-12, atol=0)
    assert np.allclose(coarse_sum, ca, rtol=1e-12, atol=0)
    assert abs(fa.sum() - 1.0) < 1e-12


def _l2_coeffs(m, g, deg, u):
    """Coefficients of the L2 projection of u onto P_deg of each cell (exact for polynomials of degree <= deg)."""
    nb = n_basis(deg)
    out = np.zeros(m.n_elem * nb)
    for e in range(m.n_elem):
        pts, w = polygon_rule(m.polygon(e), deg + 3)
        v, _ = eval_basis(deg, g.bbox[e], pts)
        M = np.einsum("q,qa,qb->ab", w, v, v)
        out[e * nb:(e + 1) * nb] = np.linalg.solve(M, np.einsum("q,qa,q->a", w, v, u(pts)))
    return out


@pytest.mark.parametrize("p,q", [(1, 1), (2, 1), (3, 2), (3, 3)])
def test_global_polynomials_are_reproduced(p, q):
    fm, fg, cm, cg = _pair(90, 13)
    R0T = schwarz.prolongation_nonnested(fm, fg, cm, cg, p, q)
    polys = [lambda X: np.ones(len(X)), lambda X: 1.0 + 2.0 * X[:, 0] - 3.0 * X[:, 1]]
    if q >= 2:
        polys.append(lambda X: X[:, 0] * X[:, 1] - 0.5 * X[:, 1] ** 2)
    if q >= 3:
        polys.append(lambda X: X[:, 0] ** 3 - X[:, 0] * X[:, 1] ** 2)
    for u in polys:
        c = _l2_coeffs(cm, cg, q, u)
        f = _l2_coeffs(fm, fg, p, u)
        assert np.linalg.norm(R0T @ c - f) <= 1e-11 * np.linalg.norm(f)


@pytest.mark.parametrize("p,q", [(2, 1), (3, 3)])
def test_same_mesh_gives_the_nested_injection(p, q):
    fm = mesh(60, 5)
    fg = build_geometry(fm)
    nn = schwarz.prolongation_nonnested(fm, fg, fm, fg, p, q)
    nested = schwarz.prolongation(fm, fg, np.arange(fm.n_elem), p, q)
    assert abs(nn - nested).max() <= 1e-12 * abs(nested).max()


def test_nonnested_schwarz_is_spd_and_pcg_converges():
    fm, fg, cm, cg = _pair(100, 9)
    p, q = 2, 1
    A, b, g = sipg.assemble(fm, np.ones(fm.n_elem), p, 10.0, f_sin)
    sub = partition.subdomains(g.centroid, 4)
    O = schwarz.build(A, fm, g, p, sub, None, q, coarse=(cm, cg))
    assert O.R0T.shape == (fm.n_elem * n_basis(p), cm.n_elem * n_basis(q))
    B = O.dense(A.shape[0])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    res = pcg.pcg(A, b, O.apply, rtol=1e-10)
    xs = spla.spsolve(A.tocsc(), b)
    assert res.converged and np.linalg.norm(res.x - xs) <= 1e-8 * np.linalg.norm(xs)
