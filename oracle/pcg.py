"""Additive Schwarz preconditioned conjugate gradients (ASPCG, Sec. 7).

Hestenes-Stiefel PCG from the zero initial guess.  Stop test: the Euclidean norm of the (recursively
updated, unpreconditioned) residual relative to ||b||_2 drops below rtol (Sec. 7 uses 1e-8).  The
condition number K(P_ad) is estimated from the CG coefficients through the Lanczos tridiagonal
matrix T_k with T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1} (beta_{-1}/alpha_{-1} = 0) and
T_{j,j+1} = sqrt(beta_j)/alpha_j; its extreme eigenvalues approximate those of B A.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    converged: bool
    alphas: list = field(default_factory=list)
    betas: list = field(default_factory=list)
    resid: list = field(default_factory=list)   # ||r_k|| / ||b||, k = 0..iters


def pcg(A, b: np.ndarray, apply_B, rtol: float = 1e-8, maxit: int = 10000, fixed_iters=None) -> PCGResult:
    """If ``fixed_iters`` is given, exactly that many iterations run (no stop test)."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    res = PCGResult(x=x, iters=0, converged=False, resid=[1.0 if bnorm > 0 else 0.0])
    if bnorm == 0.0:
        res.converged = True
        return res
    z = apply_B(r)
    p = z.copy()
    gamma = float(r @ z)
    limit = maxit if fixed_iters is None else fixed_iters
    k = 0
    while k < limit:
        q = A @ p
        alpha = gamma / float(p @ q)
        x += alpha * p
        r -= alpha * q
        k += 1
        res.alphas.append(alpha)
        rel = np.linalg.norm(r) / bnorm
        res.resid.append(rel)
        if fixed_iters is None and rel <= rtol:
            res.converged = True
            break
        z = apply_B(r)
        gamma_new = float(r @ z)
        beta = gamma_new / gamma
        res.betas.append(beta)
        p = z + beta * p
        gamma = gamma_new
    res.x = x
    res.iters = k
    if fixed_iters is not None:
        res.converged = res.resid[-1] <= rtol
    return res


def lanczos_extremes(alphas, betas):
    """(lambda_min, lambda_max) of the Lanczos tridiagonal built from k CG steps."""
    k = len(alphas)
    if k == 0:
        return float("nan"), float("nan")
    d = np.empty(k)
    e = np.empty(max(k - 1, 0))
    for j in range(k):
        d[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j < k - 1:
            e[j] = np.sqrt(betas[j]) / alphas[j]
    ev = sla.eigvalsh_tridiagonal(d, e) if k > 1 else d
    return float(ev.min()), float(ev.max())


def condition_estimate(res: PCGResult) -> float:
    lo, hi = lanczos_extremes(res.alphas, res.betas[:max(len(res.alphas) - 1, 0)])
    return hi / lo
