"""Quadrature rules, derived from the mathematics (no tables).

The paper fixes no quadrature.  Element integrals use a fan of triangles from the polygon's
vertex average, each integrated by a Duffy-collapsed tensor Gauss-Legendre rule; face integrals
use Gauss-Legendre on the segment.  With m points per direction the Duffy rule integrates
polynomials of total degree 2m - 2 exactly, so m = p + 2 makes every SIPG matrix entry exact.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_legendre(m: int):
    """Nodes and weights of the m-point Gauss-Legendre rule on [-1, 1].

    Newton iteration on P_m, evaluated with the three-term recurrence
    (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}, with P_m'(t) = m (t P_m - P_{m-1}) / (t^2 - 1);
    the weights are 2 / ((1 - t^2) P_m'(t)^2).
    """
    if m == 1:
        return np.array([0.0]), np.array([2.0])

    def legendre_pair(t):
        """(P_m(t), P_{m-1}(t))."""
        p_prev, p_cur = 1.0, t
        for k in range(1, m):
            p_prev, p_cur = p_cur, ((2 * k + 1) * t * p_cur - k * p_prev) / (k + 1)
        return p_cur, p_prev

    nodes = np.empty(m)
    weights = np.empty(m)
    for i in range(m):
        t = math.cos(math.pi * (i + 0.75) / (m + 0.5))
        for _ in range(100):
            pm, pm1 = legendre_pair(t)
            dp = m * (t * pm - pm1) / (t * t - 1.0)
            dt = pm / dp
            t -= dt
            if abs(dt) < 1e-16:
                break
        pm, pm1 = legendre_pair(t)
        dp = m * (t * pm - pm1) / (t * t - 1.0)
        nodes[i] = t
        weights[i] = 2.0 / ((1.0 - t * t) * dp * dp)
    order = np.argsort(nodes)
    return nodes[order], weights[order]


def gauss_legendre_01(m: int):
    t, w = gauss_legendre(m)
    return 0.5 * (t + 1.0), 0.5 * w


def triangle_rule(a, b, c, m: int):
    """Duffy-collapsed rule on triangle (a, b, c): P(u, v) = a + u (b - a) + u v (c - b),
    dA = u |det(b - a, c - b)| du dv on the unit square."""
    a, b, c = (np.asarray(v, dtype=np.float64) for v in (a, b, c))
    u, wu = gauss_legendre_01(m)
    v, wv = gauss_legendre_01(m)
    e1 = b - a
    e2 = c - b
    jac = abs(e1[0] * e2[1] - e1[1] * e2[0])
    pts = []
    wts = []
    for i in range(m):
        for j in range(m):
            pts.append(a + u[i] * e1 + u[i] * v[j] * e2)
            wts.append(wu[i] * wv[j] * u[i] * jac)
    return np.array(pts), np.array(wts)


def polygon_rule(poly: np.ndarray, m: int):
    """Fan of triangles (vertex average, v_k, v_{k+1}) for a polygon given by its vertices."""
    poly = np.asarray(poly, dtype=np.float64)
    centre = poly.mean(axis=0)
    pts, wts = [], []
    n = len(poly)
    for k in range(n):
        p, w = triangle_rule(centre, poly[k], poly[(k + 1) % n], m)
        pts.append(p)
        wts.append(w)
    return np.concatenate(pts), np.concatenate(wts)


def segment_rule(a, b, m: int):
    """Gauss-Legendre points on the segment from a to b; weights include the length."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    t, w = gauss_legendre_01(m)
    length = math.hypot(*(b - a))
    return a[None, :] + t[:, None] * (b - a)[None, :], w * length
