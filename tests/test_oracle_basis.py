"""Pins for the oracle basis: orthonormality on the box (closed form), span of P_p, derivatives."""
import numpy as np
import pytest

from oracle.basis import eval_basis, index_pairs, legendre_table, n_basis
from oracle.quadrature import gauss_legendre


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_orthonormal_on_box(p):
    box = (0.3, 0.75, -0.2, 0.1)
    t, w = gauss_legendre(p + 2)
    xs = box[0] + (box[1] - box[0]) * 0.5 * (t + 1)
    ys = box[2] + (box[3] - box[2]) * 0.5 * (t + 1)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    W = np.outer(w, w) * 0.25 * (box[1] - box[0]) * (box[3] - box[2])
    v, _ = eval_basis(p, box, np.stack([X.ravel(), Y.ravel()], 1))
    G = v.T @ (W.ravel()[:, None] * v)
    assert np.abs(G - np.eye(n_basis(p))).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_spans_total_degree_space(p):
    rng = np.random.default_rng(p)
    pts = rng.uniform(0, 1, (60, 2))
    v, _ = eval_basis(p, (0, 1, 0, 1), pts)
    mono = np.stack([pts[:, 0] ** i * pts[:, 1] ** j for (i, j) in index_pairs(p)], 1)
    assert np.linalg.matrix_rank(v) == n_basis(p)
    # each basis function is a polynomial of total degree <= p: it lies in the monomial span
    coef, *_ = np.linalg.lstsq(mono, v, rcond=None)
    assert np.abs(mono @ coef - v).max() < 1e-10


def test_ordering():
    assert index_pairs(2) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    assert n_basis(3) == 10 and n_basis(4) == 15


def test_legendre_against_numpy():
    t = np.linspace(-1, 1, 11)
    L, dL = legendre_table(7, t)
    for k in range(8):
        c = np.zeros(k + 1)
        c[k] = 1
        assert np.allclose(L[k], np.polynomial.legendre.legval(t, c), atol=1e-14)
        assert np.allclose(dL[k], np.polynomial.legendre.legval(t, np.polynomial.legendre.legder(c)), atol=1e-12)


def test_gradient_matches_finite_difference():
    box = (0.1, 0.4, 0.2, 0.9)
    pts = np.array([[0.2, 0.5], [0.35, 0.3]])
    _, g = eval_basis(3, box, pts)
    h = 1e-6
    for d in range(2):
        e = np.zeros(2)
        e[d] = h
        vp, _ = eval_basis(3, box, pts + e)
        vm, _ = eval_basis(3, box, pts - e)
        assert np.allclose(g[:, :, d], (vp - vm) / (2 * h), atol=1e-6 * np.abs(g).max())
