#!/usr/bin/env python
"""Writes the oracle's converged solves of the full-size workloads into tests/golden/oracle_solve_*.txt.

Only ``oracle/`` (and the seeded input generators in ``synth/``) are called here: no value comes from the
CUDA library.  One file per case: the 16384-cell Lloyd-Voronoi mesh (seed 2), 64 RCB subdomains, 256 RCB
agglomerates at q = 1, rho = contrast on the odd cells of a 4 x 4 checkerboard of subdomains,
f = 2 pi^2 sin(pi x) sin(pi y), ASPCG from x = 0 to ||r_k|| <= 1e-8 ||b|| (Sec. 7).  Each file holds the
oracle's iteration count, its recursive and true relative residuals, the Lanczos K estimate, ||b||, ||x||,
lambda_min(A) (shift-invert Lanczos, for the a-posteriori error bound ||x - x*|| <= ||b - A x|| / lambda_min)
and the entries of b and x at 1000 evenly spaced dofs.

Usage: python tests/golden/make_oracle_solutions.py [case ...]   (cases: p3_c1e4, p4_c1, p4_c1e2, p4_c1e4, p4_c1e6)
Run time on 8 x86 cores: about 10 minutes for p3_c1e4 and 20-30 minutes per p = 4 case.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_ELEM, SEED, NSUB, NCOARSE, Q = 16384, 2, 64, 256, 1
N_SAMPLES = 1000
CASES = {"p3_c1e4": (3, 1e4), "p4_c1": (4, 1.0), "p4_c1e2": (4, 1e2), "p4_c1e4": (4, 1e4), "p4_c1e6": (4, 1e6)}


def f_sin(X):
    return 2 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])


def sample_indices(ndof: int) -> np.ndarray:
    return np.unique(np.linspace(0, ndof - 1, N_SAMPLES).round().astype(np.int64))


def path_of(case: str) -> str:
    return os.path.join(HERE, f"oracle_solve_16384cells_{case}.txt")


def run(case: str) -> None:
    import scipy.sparse.linalg as spla

    from oracle import partition, pcg, schwarz, sipg
    from oracle.geometry import build_geometry
    from synth.coeff import checker_per_subdomain
    from synth.voronoi import voronoi_mesh

    p, contrast = CASES[case]
    t0 = time.time()
    m = voronoi_mesh(N_ELEM, SEED)
    g = build_geometry(m)
    sub = partition.subdomains(g.centroid, NSUB)
    agg = partition.agglomerates(g.centroid, sub, NSUB, NCOARSE)
    rho = checker_per_subdomain(m, sub, contrast)
    A, b, _ = sipg.assemble(m, rho, p, 10.0, f_sin, geom=g)
    A = A.tocsr()
    O = schwarz.build(A, m, g, p, sub, agg, Q)
    t1 = time.time()
    res = pcg.pcg(A, b, O.apply, rtol=1e-8)
    t2 = time.time()
    x = res.x
    bn = float(np.linalg.norm(b))
    true_rr = float(np.linalg.norm(b - A @ x) / bn)
    kappa = pcg.condition_estimate(res)
    lam_min = float(spla.eigsh(A, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0])
    idx = sample_indices(A.shape[0])
    with open(path_of(case), "w") as f:
        f.write(f"# Oracle ASPCG solve (Sec. 7: zero initial guess, stop at ||r_k|| <= 1e-8 ||b||, Lanczos K from the CG\n")
        f.write(f"# coefficients) of the 16384-cell Lloyd-Voronoi mesh (seed 2), SIPG p = {p} (C_sigma = 10, Sec. 2),\n")
        f.write(f"# 64 RCB subdomains, 256 RCB agglomerates at q = 1 (Sec. 3), rho = {contrast:g} on the odd cells of a 4 x 4\n")
        f.write("# checkerboard of subdomains, f = 2 pi^2 sin(pi x) sin(pi y).  Written by tests/golden/make_oracle_solutions.py,\n")
        f.write("# which calls only oracle/ and synth/.  lambda_min: smallest eigenvalue of A (shift-invert Lanczos).\n")
        f.write(f"p {p}\ncontrast {contrast!r}\nndof {A.shape[0]}\niters {res.iters}\nconverged {int(res.converged)}\n")
        f.write(f"relres {float(res.resid[-1])!r}\ntrue_relres {true_rr!r}\nkappa {float(kappa)!r}\nbnorm {bn!r}\n")
        f.write(f"xnorm {float(np.linalg.norm(x))!r}\nlambda_min {lam_min!r}\n")
        f.write(f"setup_seconds {t1 - t0:.1f}\nsolve_seconds {t2 - t1:.1f}\n")
        f.write("# samples: dof b x\n")
        for i in idx:
            f.write(f"s {int(i)} {float(b[i])!r} {float(x[i])!r}\n")
    print(f"{case}: {res.iters} iterations, true relres {true_rr:.3e}, K {kappa:.1f}, setup {t1 - t0:.0f} s, "
          f"solve {t2 - t1:.0f} s", flush=True)


def load(case: str) -> dict:
    """The stored solve of one case: scalars by name, and 'idx', 'b', 'x' arrays of the sampled dofs."""
    out = {}
    idx, bs, xs = [], [], []
    with open(path_of(case)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "s":
                idx.append(int(parts[1]))
                bs.append(float(parts[2]))
                xs.append(float(parts[3]))
            else:
                v = parts[1]
                if v.startswith("np.float64("):   # numpy 2 repr of a float64 scalar
                    v = v[len("np.float64("):-1]
                out[parts[0]] = float(v)
    out["idx"] = np.array(idx, dtype=np.int64)
    out["b"] = np.array(bs)
    out["x"] = np.array(xs)
    return out


if __name__ == "__main__":
    for c in (sys.argv[1:] or list(CASES)):
        run(c)
