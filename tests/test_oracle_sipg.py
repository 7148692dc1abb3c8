"""Pins for the oracle's SIPG assembly (Sec. 2, Eq. Ah, Eq. lifting, Eq. Sigma).

* hand-derived entries on a two-square mesh (closed forms below) pin the penalty with the harmonic
  average of rho, the consistency factor <rho>/2 and the boundary terms; a square next to a 2 x 1
  rectangle pins the harmonic average of h (Sec. 2 defines <.> for both);
* symmetry and positive definiteness (Lemma 5.1: coercive for C_sigma large enough);
* consistency: u = x(1-x)y(1-y) lies in P_4 and vanishes on the boundary, so for p >= 4 the SIPG
  solution reproduces it to rounding;
* convergence: ||u - u_h||_L2 = O(h^{p+1}) for u = sin(pi x) sin(pi y), the textbook SIPG rate.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import error, sipg
from oracle.basis import n_basis
from oracle.geometry import build_geometry
from synth.voronoi import PolyMesh, quad_mesh, voronoi_mesh


def two_squares():
    xy = np.array([[0, 0], [1, 0], [2, 0], [2, 1], [1, 1], [0, 1]], float)
    return PolyMesh(xy=xy, poly_ptr=np.array([0, 4, 8], np.int32),
                    poly_vtx=np.array([0, 1, 4, 5, 1, 2, 3, 4], np.int32))


def test_two_square_entries_closed_form():
    """kappa_1 = [0,1]^2 (rho 1), kappa_2 = [1,2]x[0,1] (rho 3), p = 1, C_sigma = 10.
    Basis per box: phi_0 = 1, phi_1 = sqrt3 xi, phi_2 = sqrt3 eta.  h = sqrt2 for both, so
    <h> = sqrt2, <rho> = 2*1*3/4 = 3/2, sigma_I = 10 * 3/2 / sqrt2, sigma_B1 = 10 / sqrt2,
    sigma_B2 = 30 / sqrt2.  Derivations (interior face x = 1, n = (1, 0), kappa^+ = kappa_1):
      A[1.phi0, 2.phi0] = sigma_I * (+1)(-1)                                  = -sigma_I
      A[1.phi0, 2.phi1] = -<rho>/2 * 2sqrt3 + sigma_I * (-1)(-sqrt3)          = sqrt3 (sigma_I - 3/2)
      A[1.phi1, 2.phi1] = -<rho>/2*sqrt3*2sqrt3 - <rho>/2*(-1)(-sqrt3)(2sqrt3) + 3 sigma_I = 3 sigma_I - 9
      A[1.phi2, 2.phi2] = -sigma_I * int_0^1 3 (2y-1)^2 dy                   = -sigma_I
      A[1.phi1, 1.phi1] = 12 (element) + (-12 + 3 sigma_B1) (x = 0) + (-9 + 3 sigma_I) (x = 1)
                          + sigma_B1 (y = 0) + sigma_B1 (y = 1)               = 5 sigma_B1 + 3 sigma_I - 9
      A[2.phi0, 2.phi0] = sigma_I + 3 sigma_B2
    """
    mesh = two_squares()
    A, _, _ = sipg.assemble(mesh, np.array([1.0, 3.0]), 1, 10.0)
    A = A.toarray()
    s3 = math.sqrt(3.0)
    sI = 15.0 / math.sqrt(2.0)
    sB1 = 10.0 / math.sqrt(2.0)
    sB2 = 30.0 / math.sqrt(2.0)
    d = lambda e, a: 3 * e + a  # noqa: E731
    expect = {
        (d(0, 0), d(1, 0)): -sI,
        (d(0, 0), d(1, 1)): s3 * (sI - 1.5),
        (d(0, 1), d(1, 1)): 3 * sI - 9.0,
        (d(0, 2), d(1, 2)): -sI,
        (d(0, 1), d(0, 1)): 5 * sB1 + 3 * sI - 9.0,
        (d(1, 0), d(1, 0)): sI + 3 * sB2,
    }
    for (i, j), v in expect.items():
        assert A[i, j] == pytest.approx(v, rel=1e-13, abs=1e-13), (i, j)
        assert A[j, i] == pytest.approx(v, rel=1e-13, abs=1e-13), (j, i)


def test_unequal_cells_penalty_uses_harmonic_h():
    """kappa_1 = [0,1]^2, kappa_2 = [1,3]x[0,1], rho = 1, p = 1, C_sigma = 10.  h_1 = sqrt2, h_2 = sqrt5, so
    <h> = 2 sqrt2 sqrt5 / (sqrt2 + sqrt5) and sigma_I = 10 / <h>; sigma_B2 = 10 / sqrt5.  phi_0 = 1 on kappa_1
    and 1/sqrt2 on kappa_2 (box 2 x 1), with zero gradient, so only penalty terms reach these entries:
      A[1.phi0, 2.phi0] = sigma_I (+1)(-1) int_0^1 1 * (1/sqrt2) dy           = -sigma_I / sqrt2
      A[2.phi0, 2.phi0] = sigma_I / 2 (face x = 1) + sigma_B2 / 2 * (1 + 2 + 2) = sigma_I / 2 + 5 sqrt5
    (the arithmetic mean or the larger of h_1, h_2 in place of <h> changes both)."""
    xy = np.array([[0, 0], [1, 0], [3, 0], [3, 1], [1, 1], [0, 1]], float)
    mesh = PolyMesh(xy=xy, poly_ptr=np.array([0, 4, 8], np.int32),
                    poly_vtx=np.array([0, 1, 4, 5, 1, 2, 3, 4], np.int32))
    A = sipg.assemble(mesh, np.ones(2), 1, 10.0)[0].toarray()
    r2, r5 = math.sqrt(2.0), math.sqrt(5.0)
    sI = 10.0 * (r2 + r5) / (2.0 * r2 * r5)
    assert A[0, 3] == pytest.approx(-sI / r2, rel=1e-13)
    assert A[3, 0] == pytest.approx(-sI / r2, rel=1e-13)
    assert A[3, 3] == pytest.approx(sI / 2.0 + 5.0 * r5, rel=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_symmetric_positive_definite(p):
    mesh = voronoi_mesh(24, 11, lloyd=5)
    rho = np.where(np.arange(24) % 3 == 0, 1e3, 1.0)
    A, _, _ = sipg.assemble(mesh, rho, p, 10.0)
    A = A.toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_polynomial_solution_reproduced_p4():
    mesh = voronoi_mesh(20, 5, lloyd=10)
    p = 4
    u = lambda X: X[:, 0] * (1 - X[:, 0]) * X[:, 1] * (1 - X[:, 1])  # noqa: E731
    f = lambda X: 2.0 * (X[:, 0] * (1 - X[:, 0]) + X[:, 1] * (1 - X[:, 1]))  # noqa: E731
    A, b, geom = sipg.assemble(mesh, np.ones(mesh.n_elem), p, 10.0, f)
    x = spla.spsolve(A.tocsc(), b)
    proj = error.l2_projection(mesh, geom, p, u)
    assert np.abs(x - proj).max() <= 1e-10 * np.abs(proj).max()
    assert error.l2_error(mesh, geom, p, x, u) < 1e-12


def test_polynomial_solution_not_reproduced_p3():
    # u is degree 4: with p = 3 the error must be visibly nonzero (guards the test above)
    mesh = voronoi_mesh(20, 5, lloyd=10)
    u = lambda X: X[:, 0] * (1 - X[:, 0]) * X[:, 1] * (1 - X[:, 1])  # noqa: E731
    f = lambda X: 2.0 * (X[:, 0] * (1 - X[:, 0]) + X[:, 1] * (1 - X[:, 1]))  # noqa: E731
    A, b, geom = sipg.assemble(mesh, np.ones(mesh.n_elem), 3, 10.0, f)
    x = spla.spsolve(A.tocsc(), b)
    assert error.l2_error(mesh, geom, 3, x, u) > 1e-7


@pytest.mark.parametrize("p,sizes", [(1, (64, 256, 1024)), (2, (64, 256, 1024))])
def test_optimal_l2_rate(p, sizes):
    u = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])  # noqa: E731
    f = lambda X: 2 * np.pi ** 2 * u(X)  # noqa: E731
    hs, errs = [], []
    for n in sizes:
        mesh = voronoi_mesh(n, 100 + n)
        A, b, geom = sipg.assemble(mesh, np.ones(n), p, 10.0, f)
        x = spla.spsolve(A.tocsc(), b)
        hs.append(1.0 / math.sqrt(n))
        errs.append(error.l2_error(mesh, geom, p, x, u))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(slope - (p + 1)) < 0.3, (slope, errs)


def test_faces_euler_and_perimeter():
    mesh = voronoi_mesh(200, 3)
    g = build_geometry(mesh)
    nv = len(np.unique(mesh.poly_vtx))
    assert nv - len(g.faces) + mesh.n_elem == 1           # Euler for a disc
    bnd = [f for f in g.faces if f[1] < 0]
    per = sum(np.hypot(*(mesh.xy[b] - mesh.xy[a])) for (_, _, a, b) in bnd)
    assert per == pytest.approx(4.0, rel=1e-13)
    assert g.area.sum() == pytest.approx(1.0, rel=1e-13)
    # h_kappa is the largest vertex distance: on squares it is the diagonal
    gq = build_geometry(quad_mesh(3))
    assert np.allclose(gq.diameter, math.sqrt(2.0) / 3.0, rtol=1e-15)


def test_dofs_layout():
    mesh = quad_mesh(2)
    A, _, _ = sipg.assemble(mesh, np.ones(4), 2, 10.0)
    assert A.shape == (4 * n_basis(2),) * 2
