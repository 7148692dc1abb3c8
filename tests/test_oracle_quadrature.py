"""Pins for the oracle's quadrature: library Gauss-Legendre and exact polygon moments (Green's theorem)."""
import math

import numpy as np
import pytest

from oracle.quadrature import gauss_legendre, polygon_rule, segment_rule, triangle_rule


def polygon_moment(poly, a, b):
    """Closed form of int_P x^a y^b dA for a CCW polygon (divergence theorem applied edge by edge):
    a! b! / (a+b+2)! sum_i cross_i sum_{k<=a, l<=b} C(k+l, l) C(a+b-k-l, b-l) x_i^k x_{i+1}^{a-k} y_i^l y_{i+1}^{b-l}."""
    n = len(poly)
    total = 0.0
    for i in range(n):
        x0, y0 = poly[i]
        x1, y1 = poly[(i + 1) % n]
        cross = x0 * y1 - x1 * y0
        s = 0.0
        for k in range(a + 1):
            for l in range(b + 1):
                s += (math.comb(k + l, l) * math.comb(a + b - k - l, b - l)
                      * x0 ** k * x1 ** (a - k) * y0 ** l * y1 ** (b - l))
        total += cross * s
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2) * total


def random_convex_polygon(rng, n):
    ang = np.sort(rng.uniform(0, 2 * np.pi, n))
    rad = rng.uniform(0.5, 1.0)
    c = rng.uniform(-1, 1, 2)
    return c + rad * np.stack([np.cos(ang), np.sin(ang)], 1)


@pytest.mark.parametrize("m", range(1, 13))
def test_gauss_legendre_matches_numpy(m):
    t, w = gauss_legendre(m)
    tr, wr = np.polynomial.legendre.leggauss(m)
    assert np.allclose(t, tr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=2e-15, rtol=0)


def test_moment_formula_on_unit_square():
    sq = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    for a in range(5):
        for b in range(5):
            assert polygon_moment(sq, a, b) == pytest.approx(1.0 / ((a + 1) * (b + 1)), rel=1e-14)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6])
def test_polygon_rule_exact_up_to_degree(m):
    rng = np.random.default_rng(m)
    for _ in range(5):
        poly = random_convex_polygon(rng, int(rng.integers(3, 9)))
        pts, w = polygon_rule(poly, m)
        for a in range(2 * m - 1):
            for b in range(2 * m - 1 - a):
                exact = polygon_moment(poly, a, b)
                got = float(w @ (pts[:, 0] ** a * pts[:, 1] ** b))
                scale = polygon_moment(poly, 0, 0) * 2.0 ** (a + b)
                assert abs(got - exact) <= 1e-13 * scale, (a, b, got, exact)


def test_triangle_rule_not_exact_beyond_degree():
    # guards against a rule silently using more points than m: degree 2m must show an error
    m = 2
    pts, w = triangle_rule([0, 0], [1, 0], [0, 1], m)
    exact = polygon_moment(np.array([[0, 0], [1, 0], [0, 1]], float), 2 * m, 0)
    assert abs(float(w @ pts[:, 0] ** (2 * m)) - exact) > 1e-6


def test_segment_rule():
    pts, w = segment_rule([0.2, 0.1], [1.1, 0.7], 4)
    L = math.hypot(0.9, 0.6)
    assert w.sum() == pytest.approx(L, rel=1e-15)
    # int_0^1 t^7 dt on the parametrisation, x = 0.2 + 0.9 t
    t = (pts[:, 0] - 0.2) / 0.9
    assert float(w @ t ** 7) == pytest.approx(L / 8.0, rel=1e-14)
