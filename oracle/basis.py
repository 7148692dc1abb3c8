"""Physical-frame polynomial basis of total degree p (Sec. 2, Eq. Vh).

The paper leaves the basis open beyond building it in the physical frame.  Reading adopted:
products of Legendre polynomials on the element's axis-aligned bounding box
[x0, x1] x [y0, y1], phi_ij(x, y) = c_ij L_i(xi) L_j(eta), xi = 2 (x - xc) / wx,
eta = 2 (y - yc) / wy, i + j <= p, normalised c_ij = sqrt((2i+1)(2j+1) / (wx wy)) so that the
functions are orthonormal on the box.  Order: total degree d = i + j ascending, then i descending.
"""
from __future__ import annotations

import numpy as np


def n_basis(p: int) -> int:
    return (p + 1) * (p + 2) // 2


def index_pairs(p: int):
    """[(i, j)] in basis order."""
    out = []
    for d in range(p + 1):
        for i in range(d, -1, -1):
            out.append((i, d - i))
    return out


def legendre_table(n: int, t: np.ndarray):
    """L_0..L_n and their derivatives at points t (Bonnet recurrence; L'_{k+1} = L'_{k-1} + (2k+1) L_k)."""
    t = np.asarray(t, dtype=np.float64)
    L = np.zeros((n + 1,) + t.shape)
    dL = np.zeros((n + 1,) + t.shape)
    L[0] = 1.0
    if n >= 1:
        L[1] = t
        dL[1] = 1.0
    for k in range(1, n):
        L[k + 1] = ((2 * k + 1) * t * L[k] - k * L[k - 1]) / (k + 1)
        dL[k + 1] = dL[k - 1] + (2 * k + 1) * L[k]
    return L, dL


def eval_basis(p: int, box, pts: np.ndarray):
    """Values (npts, nb) and gradients (npts, nb, 2) of the basis on ``box`` = (x0, x1, y0, y1)."""
    x0, x1, y0, y1 = box
    wx, wy = x1 - x0, y1 - y0
    xc, yc = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
    pts = np.asarray(pts, dtype=np.float64)
    xi = 2.0 * (pts[:, 0] - xc) / wx
    eta = 2.0 * (pts[:, 1] - yc) / wy
    Lx, dLx = legendre_table(p, xi)
    Ly, dLy = legendre_table(p, eta)
    pairs = index_pairs(p)
    val = np.empty((len(pts), len(pairs)))
    grad = np.empty((len(pts), len(pairs), 2))
    for a, (i, j) in enumerate(pairs):
        c = np.sqrt((2 * i + 1) * (2 * j + 1) / (wx * wy))
        val[:, a] = c * Lx[i] * Ly[j]
        grad[:, a, 0] = c * dLx[i] * (2.0 / wx) * Ly[j]
        grad[:, a, 1] = c * Lx[i] * dLy[j] * (2.0 / wy)
    return val, grad
