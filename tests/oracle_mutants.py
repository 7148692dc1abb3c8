#!/usr/bin/env python
"""Mutation check of the oracle's pins: plants one plausible mistake at a time in a temporary copy of
oracle/ (with synth/ and tests/ beside it) and runs the CPU pins (tests/test_oracle_*.py) against it.
Every mistake must make at least one pin fail; the repository itself is never modified.

    python tests/oracle_mutants.py            # all mistakes, about 10 minutes on 8 cores
    python tests/oracle_mutants.py -k pcg     # only the mistakes planted in pcg.py

Exit status 1 if a mistake survives.  The mistakes cover every oracle module: the SIPG terms of Eq. Ah
and Eq. Sigma (averages, signs, factors, penalty scaling, quadrature order), the basis (normalisation,
recurrences, chain rule, order), the quadrature rules, the geometry, the Schwarz operator of Sec. 3 (local
solves, R_0^T of Eq. R0T, A_0 of Eq. A0, the weight of the coarse term), PCG and its stop test (Sec. 7),
the Lanczos estimate, the partitions, and the non-nested coarse space of Example 4 (clipping, the rule on
the pieces, the mass-matrix solve).
"""
from __future__ import annotations

import argparse
import importlib.util
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (oracle module, mistake, original text, planted text)
MUTANTS = [
    ("sipg.py", "harmonic average of rho -> arithmetic mean", "return 2.0 * a * b / (a + b)", "return 0.5 * (a + b)"),
    ("sipg.py", "consistency factor 1 instead of 1/2 (one term)", "blk = (-0.5 * rho_avg * sa", "blk = (-1.0 * rho_avg * sa"),
    ("sipg.py", "symmetry term with the wrong sign", "- 0.5 * rho_avg * sb", "+ 0.5 * rho_avg * sb"),
    ("sipg.py", "interior penalty p instead of p^2", "sigma = c_sigma * rho_avg * p * p / h_avg",
     "sigma = c_sigma * rho_avg * p / h_avg"),
    ("sipg.py", "larger h instead of the harmonic average", "h_avg = harmonic(geom.diameter[ep], geom.diameter[em])",
     "h_avg = max(geom.diameter[ep], geom.diameter[em])"),
    ("sipg.py", "boundary penalty without rho", "sigma = c_sigma * rho[ep] * p * p / geom.diameter[ep]",
     "sigma = c_sigma * p * p / geom.diameter[ep]"),
    ("sipg.py", "boundary consistency term dropped", "+ np.einsum(\"q,qb,qa->ab\", w, v, -rho[ep] * dn)",
     "+ 0.0 * np.einsum(\"q,qb,qa->ab\", w, v, -rho[ep] * dn)"),
    ("sipg.py", "face normal flipped", "n = np.array([d[1], -d[0]])", "n = np.array([-d[1], d[0]])"),
    ("sipg.py", "minus side without its sign", "for e, s in ((ep, 1.0), (em, -1.0)):", "for e, s in ((ep, 1.0), (em, 1.0)):"),
    ("sipg.py", "matrix quadrature m = p (inexact)", "m_mat = p + 2", "m_mat = p"),
    ("sipg.py", "stiffness without rho", "K = rho[e] * np.einsum", "K = 1.0 * np.einsum"),
    ("sipg.py", "load vector without the weights", "b[e * nb:(e + 1) * nb] = val_f.T @ (w_f * f(pts_f))",
     "b[e * nb:(e + 1) * nb] = val_f.T @ f(pts_f)"),
    ("sipg.py", "load vector with a one-point rule", "pts_f, w_f = polygon_rule(poly, p + 5)", "pts_f, w_f = polygon_rule(poly, 1)"),
    ("basis.py", "normalisation with wx twice", "c = np.sqrt((2 * i + 1) * (2 * j + 1) / (wx * wy))",
     "c = np.sqrt((2 * i + 1) * (2 * j + 1) / (wx * wx))"),
    ("basis.py", "x derivative with 1/wx", "grad[:, a, 0] = c * dLx[i] * (2.0 / wx) * Ly[j]",
     "grad[:, a, 0] = c * dLx[i] * (1.0 / wx) * Ly[j]"),
    ("basis.py", "y derivative with wx", "grad[:, a, 1] = c * Lx[i] * dLy[j] * (2.0 / wy)",
     "grad[:, a, 1] = c * Lx[i] * dLy[j] * (2.0 / wx)"),
    ("basis.py", "Legendre derivative recurrence 2k", "dL[k + 1] = dL[k - 1] + (2 * k + 1) * L[k]",
     "dL[k + 1] = dL[k - 1] + (2 * k) * L[k]"),
    ("basis.py", "Bonnet recurrence sign", "L[k + 1] = ((2 * k + 1) * t * L[k] - k * L[k - 1]) / (k + 1)",
     "L[k + 1] = ((2 * k + 1) * t * L[k] + k * L[k - 1]) / (k + 1)"),
    ("basis.py", "basis order i ascending", "for i in range(d, -1, -1):", "for i in range(0, d + 1):"),
    ("quadrature.py", "Duffy Jacobian without u", "wts.append(wu[i] * wv[j] * u[i] * jac)", "wts.append(wu[i] * wv[j] * jac)"),
    ("quadrature.py", "Duffy map with u in place of u v", "pts.append(a + u[i] * e1 + u[i] * v[j] * e2)",
     "pts.append(a + u[i] * e1 + v[j] * e2)"),
    ("quadrature.py", "Gauss weights halved", "weights[i] = 2.0 / ((1.0 - t * t) * dp * dp)",
     "weights[i] = 1.0 / ((1.0 - t * t) * dp * dp)"),
    ("quadrature.py", "segment weights without the length",
     "return a[None, :] + t[:, None] * (b - a)[None, :], w * length", "return a[None, :] + t[:, None] * (b - a)[None, :], w"),
    ("geometry.py", "diameter halved", "best = max(best, math.hypot(poly[i, 0] - poly[j, 0], poly[i, 1] - poly[j, 1]))",
     "best = max(best, 0.5 * math.hypot(poly[i, 0] - poly[j, 0], poly[i, 1] - poly[j, 1]))"),
    ("geometry.py", "centroid divisor 2 instead of 3", "return 0.5 * a2, (cx / (3.0 * a2), cy / (3.0 * a2))",
     "return 0.5 * a2, (cx / (2.0 * a2), cy / (2.0 * a2))"),
    ("geometry.py", "interior faces counted twice", "elif e < other:", "else:"),
    ("schwarz.py", "local backward solve with L instead of L^T",
     "z[idx] += sla.solve_triangular(L, y, lower=True, trans=\"T\")", "z[idx] += sla.solve_triangular(L, y, lower=True)"),
    ("schwarz.py", "local matrix reduced to its diagonal", "Ai = A[idx][:, idx].toarray()",
     "Ai = np.diag(np.diag(A[idx][:, idx].toarray()))"),
    ("schwarz.py", "R_0^T without M_kappa^-1", "blk = np.linalg.solve(M, N)", "blk = N"),
    ("schwarz.py", "coarse basis on the fine box", "psi, _ = eval_basis(q, boxes[agg[e]], pts)",
     "psi, _ = eval_basis(q, geom.bbox[e], pts)"),
    ("schwarz.py", "A_0 without A", "A0 = (R0T.T @ (A @ R0T)).toarray()", "A0 = (R0T.T @ R0T).toarray()"),
    ("schwarz.py", "coarse correction dropped", "z += self.R0T @ z0", "z += 0.0 * (self.R0T @ z0)"),
    ("schwarz.py", "coarse correction doubled", "z += self.R0T @ z0", "z += 2.0 * (self.R0T @ z0)"),
    ("pcg.py", "alpha with p.p", "alpha = gamma / float(p @ q)", "alpha = gamma / float(p @ p)"),
    ("pcg.py", "beta inverted", "beta = gamma_new / gamma", "beta = gamma / gamma_new"),
    ("pcg.py", "gamma from r.r", "gamma_new = float(r @ z)", "gamma_new = float(r @ r)"),
    ("pcg.py", "search direction from r", "p = z + beta * p", "p = r + beta * p"),
    ("pcg.py", "x updated along z", "x += alpha * p", "x += alpha * z"),
    ("pcg.py", "stop test on the preconditioned residual", "rel = np.linalg.norm(r) / bnorm",
     "rel = np.linalg.norm(apply_B(r)) / np.linalg.norm(apply_B(b))"),
    ("pcg.py", "Lanczos diagonal with alpha_j for alpha_{j-1}",
     "d[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)",
     "d[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j] if j > 0 else 0.0)"),
    ("pcg.py", "Lanczos off-diagonal without the square root", "e[j] = np.sqrt(betas[j]) / alphas[j]", "e[j] = betas[j] / alphas[j]"),
    ("partition.py", "RCB cut along the shorter side", "coord = xs if ext_x >= ext_y else ys", "coord = ys if ext_x >= ext_y else xs"),
    ("partition.py", "RCB halves for odd part counts", "nl = (len(elems) * kl) // k", "nl = len(elems) // 2"),
    ("partition.py", "equal agglomerate counts per subdomain", "ci = (i + 1) * ncoarse // nsub - i * ncoarse // nsub",
     "ci = ncoarse // nsub"),
    ("partition.py", "colouring ignores neighbours", "used = {col[j] for j in adj[i] if col[j] >= 0}", "used = set()"),
    # non-nested coarse space (Example 4)
    ("schwarz.py", "non-nested: coarse basis on the fine box", "ps, _ = eval_basis(q, cb[j], pp)",
     "ps, _ = eval_basis(q, geom.bbox[e], pp)"),
    ("schwarz.py", "non-nested: no mass-matrix solve", "blk = np.linalg.solve(M, np.einsum(\"q,qa,qc->ac\", pw, ph, ps))",
     "blk = np.einsum(\"q,qa,qc->ac\", pw, ph, ps)"),
    ("schwarz.py", "clipping keeps the outside", "if sc >= 0.0:", "if sc <= 0.0:"),
    ("schwarz.py", "non-nested: one-point rule on the pieces", "pp, pw = polygon_rule(piece, p + 2)", "pp, pw = polygon_rule(piece, 1)"),
    ("schwarz.py", "non-nested: last overlapping cell dropped", "for j in cand:", "for j in cand[:-1]:"),
]


def copy_tree(dst):
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d), ignore=shutil.ignore_patterns("__pycache__"))


def run_pins(cwd):
    tests = sorted(f"tests/{f}" for f in os.listdir(os.path.join(cwd, "tests")) if f.startswith("test_oracle_"))
    cmd = [sys.executable, "-m", "pytest", *tests, "-q", "-x", "-m", "not gpu", "-p", "no:cacheprovider"]
    if importlib.util.find_spec("xdist") is not None:
        cmd += ["-n", str(min(8, os.cpu_count() or 1))]
    r = subprocess.run(cmd, cwd=cwd, capture_output=True, text=True)
    failed = [line.split(" ")[1] for line in r.stdout.splitlines() if line.startswith("FAILED")]
    return r.returncode, failed


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("-k", default="", help="only mistakes whose module or description contains this text")
    args = ap.parse_args()
    chosen = [m for m in MUTANTS if args.k in m[0] or args.k in m[1]]
    survived = 0
    with tempfile.TemporaryDirectory() as base:
        clean = os.path.join(base, "clean")
        copy_tree(clean)
        rc, failed = run_pins(clean)
        if rc != 0:
            print(f"the unmodified oracle fails its pins: {failed}")
            return 1
        for i, (mod, what, old, new) in enumerate(chosen):
            work = os.path.join(base, f"m{i}")
            copy_tree(work)
            path = os.path.join(work, "oracle", mod)
            src = open(path).read()
            if src.count(old) != 1:
                print(f"{what}: the original text occurs {src.count(old)} times in {mod}; update this list")
                return 1
            open(path, "w").write(src.replace(old, new))
            t = time.time()
            rc, failed = run_pins(work)
            survived += rc == 0
            print(f"{mod:14s} {what:48s} {'caught' if rc else 'SURVIVED'} {time.time() - t:6.1f} s  {failed[:1]}",
                  flush=True)
            shutil.rmtree(work)
    print(f"{len(chosen) - survived} of {len(chosen)} planted mistakes caught")
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main())
