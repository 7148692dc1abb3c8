"""Pins for the oracle's partitions, local/coarse spaces, preconditioner and PCG (Sec. 3, 6, 7)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import partition, pcg, schwarz, sipg
from oracle.basis import eval_basis, n_basis
from oracle.geometry import build_geometry
from synth.voronoi import quad_mesh, voronoi_mesh


def setup_problem(n=48, p=2, nsub=4, ncoarse=8, q=1, seed=7, rho=None):
    mesh = voronoi_mesh(n, seed, lloyd=10)
    rho = np.ones(n) if rho is None else rho
    A, _, geom = sipg.assemble(mesh, rho, p, 10.0)
    sub = partition.subdomains(geom.centroid, nsub)
    agg = partition.agglomerates(geom.centroid, sub, nsub, ncoarse) if ncoarse else None
    S = schwarz.build(A, mesh, geom, p, sub, agg, q)
    return mesh, geom, A, sub, agg, S


def test_rcb_quadrants_on_grid():
    g = build_geometry(quad_mesh(8))
    sub = partition.subdomains(g.centroid, 4)
    cx, cy = g.centroid[:, 0], g.centroid[:, 1]
    expect = 2 * (cx > 0.5) + (cy > 0.5)
    assert np.array_equal(sub, expect)
    agg = partition.agglomerates(g.centroid, sub, 4, 16)
    # 16 agglomerates = 2x2 blocks of the 8x8 grid, nested in the quadrants
    blocks = {}
    for e in range(64):
        key = (int(cx[e] * 4), int(cy[e] * 4))
        blocks.setdefault(key, set()).add(int(agg[e]))
    assert all(len(v) == 1 for v in blocks.values()) and len(blocks) == 16
    for j in range(16):
        assert len(set(sub[agg == j])) == 1


def test_rcb_counts():
    g = build_geometry(voronoi_mesh(300, 2, lloyd=3))
    sub = partition.subdomains(g.centroid, 7)
    counts = np.bincount(sub)
    assert counts.sum() == 300 and counts.max() - counts.min() <= 1
    agg = partition.agglomerates(g.centroid, sub, 7, 20)
    assert agg.max() + 1 == 20
    for j in range(20):
        assert len(set(sub[agg == j])) == 1
    coarse_global = partition.agglomerates(g.centroid, np.arange(300), 300, 5)
    assert np.bincount(coarse_global).tolist() == [60] * 5


def test_local_factor_is_principal_submatrix():
    _, _, A, sub, _, S = setup_problem()
    Ad = A.toarray()
    for idx, L in zip(S.local_dofs, S.local_chol):
        assert np.allclose(L @ L.T, Ad[np.ix_(idx, idx)], rtol=1e-13, atol=1e-12 * np.abs(Ad).max())


def test_prolongation_is_injection():
    """Remark 3.1: for nested spaces R_0^T v_0 = v_0 pointwise."""
    mesh, geom, _, _, agg, S = setup_problem(p=3, q=2)
    nb, nq = n_basis(3), n_basis(2)
    boxes = schwarz.agglomerate_boxes(mesh, agg, geom)
    R = S.R0T.toarray()
    rng = np.random.default_rng(0)
    for e in range(mesh.n_elem):
        poly = mesh.polygon(e)
        w = rng.dirichlet(np.ones(len(poly)), 6)
        pts = w @ poly
        phi, _ = eval_basis(3, geom.bbox[e], pts)
        psi, _ = eval_basis(2, boxes[agg[e]], pts)
        blk = R[e * nb:(e + 1) * nb, agg[e] * nq:(agg[e] + 1) * nq]
        assert np.abs(phi @ blk - psi).max() < 1e-11 * np.abs(psi).max()


def test_prolongation_q_equals_p_single_element_is_identity():
    mesh = voronoi_mesh(1, 0, lloyd=0)
    geom = build_geometry(mesh)
    R = schwarz.prolongation(mesh, geom, np.zeros(1, np.int32), 2, 2).toarray()
    assert np.abs(R - np.eye(6)).max() < 1e-12


def test_schwarz_projections_idempotent_and_spectrum():
    """P_i = R_i^T A_i^{-1} R_i A and P_0 are A-orthogonal projections; non-adjacent subdomains are
    A-orthogonal (Lemma decVi), so lambda_max(B A) <= 1 + (number of colours) (Sec. 6)."""
    mesh, geom, A, sub, agg, S = setup_problem(n=40, p=1, nsub=6, ncoarse=6)
    Ad = A.toarray()
    n = Ad.shape[0]
    for idx, L in zip(S.local_dofs, S.local_chol):
        E = np.zeros((n, len(idx)))
        E[idx, np.arange(len(idx))] = 1
        P = E @ sla.cho_solve((L, True), E.T @ Ad)
        assert np.abs(P @ P - P).max() < 1e-9
    R = S.R0T.toarray()
    P0 = R @ np.linalg.solve(S.A0, R.T @ Ad)
    assert np.abs(P0 @ P0 - P0).max() < 1e-9
    B = S.dense(n)
    ev = np.linalg.eigvals(B @ Ad)
    assert np.abs(ev.imag).max() < 1e-8 * np.abs(ev.real).max()
    adj = partition.subdomain_adjacency(sub, geom.faces)
    ncol = int(partition.greedy_colouring(adj).max()) + 1
    assert ev.real.min() > 0
    assert ev.real.max() <= 1 + ncol + 1e-9


def test_one_subdomain_no_coarse_one_iteration():
    mesh, geom, A, sub, _, S = setup_problem(nsub=1, ncoarse=0)
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    res = pcg.pcg(A, b, S.apply, rtol=1e-8)
    assert res.iters == 1 and res.converged


def test_one_subdomain_with_coarse_space_spectrum():
    """One subdomain covering the mesh: A_1 = A, so B A = P_0 + I (Sec. 3) with P_0 the A-orthogonal projection
    onto V_0.  Its spectrum is exactly 2 on V_0 (n0 times) and 1 elsewhere, and PCG ends after two iterations
    (two distinct eigenvalues); a coarse term with any other weight moves the upper eigenvalue."""
    _, _, A, _, _, S = setup_problem(n=40, p=2, nsub=1, ncoarse=8, q=1)
    Ad = A.toarray()
    n, n0 = Ad.shape[0], S.A0.shape[0]
    ev = np.sort(np.linalg.eigvals(S.dense(n) @ Ad).real)
    assert np.abs(ev[:n - n0] - 1.0).max() < 1e-9
    assert np.abs(ev[n - n0:] - 2.0).max() < 1e-9
    b = np.random.default_rng(3).standard_normal(n)
    res = pcg.pcg(A, b, S.apply, rtol=1e-8)
    assert res.converged and res.iters == 2


def test_stop_test_on_the_unpreconditioned_residual():
    """Sec. 7 stops when the Euclidean norm of the residual b - A x, relative to ||b||, drops below the tolerance:
    the recorded residual history is that of b - A x_k (the recursive residual agrees with the true one far above
    rounding here), the last entry is the first below rtol, and the iterate before it is still above."""
    _, _, A, _, _, S = setup_problem(n=48, p=2, nsub=4, ncoarse=8)
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    rtol = 1e-6
    res = pcg.pcg(A, b, S.apply, rtol=rtol)
    true_rel = lambda x: np.linalg.norm(b - A @ x) / np.linalg.norm(b)  # noqa: E731
    assert res.converged and res.resid[-1] <= rtol < res.resid[-2]
    assert true_rel(res.x) == pytest.approx(res.resid[-1], rel=1e-6)
    prev = pcg.pcg(A, b, S.apply, fixed_iters=res.iters - 1)
    assert true_rel(prev.x) == pytest.approx(res.resid[-2], rel=1e-6)


def test_pcg_matches_direct_solve():
    _, _, A, _, _, S = setup_problem(n=32, p=2, nsub=4, ncoarse=8)
    b = np.random.default_rng(2).standard_normal(A.shape[0])
    res = pcg.pcg(A, b, S.apply, rtol=1e-12)
    x = np.linalg.solve(A.toarray(), b)
    assert res.converged
    assert np.linalg.norm(res.x - x) <= 1e-9 * np.linalg.norm(x)


def test_lanczos_estimate_matches_dense_condition():
    _, _, A, _, _, S = setup_problem(n=40, p=1, nsub=5, ncoarse=5)
    Ad = A.toarray()
    b = np.random.default_rng(3).standard_normal(Ad.shape[0])
    res = pcg.pcg(A, b, S.apply, rtol=1e-10)
    ev = np.linalg.eigvals(S.dense(Ad.shape[0]) @ Ad).real
    K = ev.max() / ev.min()
    assert pcg.condition_estimate(res) == pytest.approx(K, rel=0.01)


def test_lanczos_on_known_spectrum():
    lam = np.linspace(1.0, 50.0, 30)
    A = np.diag(lam)
    res = pcg.pcg(A, np.ones(30), lambda r: r.copy(), rtol=1e-13)
    lo, hi = pcg.lanczos_extremes(res.alphas, res.betas[:len(res.alphas) - 1])
    assert lo == pytest.approx(1.0, rel=1e-8) and hi == pytest.approx(50.0, rel=1e-8)


def test_fixed_iterations_mode():
    _, _, A, _, _, S = setup_problem(n=32, p=1)
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    r1 = pcg.pcg(A, b, S.apply, rtol=1e-8)
    r2 = pcg.pcg(A, b, S.apply, fixed_iters=r1.iters)
    assert np.array_equal(r1.x, r2.x) and r2.iters == r1.iters
