#!/usr/bin/env python
"""Mutation check of the library's host C++: plants one plausible mistake at a time in a temporary copy of the
package's sources, rebuilds libdgasm.so there and runs the CPU tests of the host logic
(tests/test_library_host.py) against it.  Every mistake must make at least one of them fail; the repository
itself is never modified.  The device kernels are checked by the GPU parity tests instead.

    python tests/library_mutants.py            # all mistakes, about 30 s each (one rebuild per mistake)
    python tests/library_mutants.py -k coarse  # only those planted in coarse_nn.cpp

Exit status 1 if a mistake survives.
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1903_11357_gb300"

# (source file under csrc/, mistake, original text, planted text)
MUTANTS = [
    ("assemble.cpp", "harmonic average of rho -> arithmetic mean",
     "double rh = 2.0 * m.rho[ep] * m.rho[em] / (m.rho[ep] + m.rho[em]);", "double rh = 0.5 * (m.rho[ep] + m.rho[em]);"),
    ("assemble.cpp", "larger h instead of the harmonic average",
     "double hh = 2.0 * m.diam[ep] * m.diam[em] / (m.diam[ep] + m.diam[em]);",
     "double hh = std::max(m.diam[ep], m.diam[em]);"),
    ("assemble.cpp", "boundary penalty without rho", "double sigma = c_sigma * m.rho[e] * p * p / m.diam[e];",
     "double sigma = c_sigma * p * p / m.diam[e];"),
    ("assemble.cpp", "minus side without its sign", "double sa = (e == ep) ? 1.0 : -1.0, sb = -sa;",
     "double sa = 1.0, sb = -sa;"),
    ("assemble.cpp", "stiffness without rho", "double wr = wts[qp] * m.rho[e];", "double wr = wts[qp];"),
    ("coarse_nn.cpp", "non-nested: coarse basis on the fine box", "values(Bq, cb, cc, W.U);", "values(Bq, fb, cc, W.U);"),
    ("coarse_nn.cpp", "non-nested: clipping keeps the outside", "if (sc >= 0.0) {", "if (sc <= 0.0) {"),
    ("coarse_nn.cpp", "non-nested: piece rule one point short", "gauss_legendre01((p + q + 3) / 2, R.tN, R.wN);",
     "gauss_legendre01((p + q + 1) / 2, R.tN, R.wN);"),
    ("coarse_nn.cpp", "non-nested: mass rule one point short", "gauss_legendre01(p + 1, R.tM, R.wM);",
     "gauss_legendre01(p, R.tM, R.wM);"),
    ("coarse_nn.cpp", "non-nested: backward solve skipped", "for (int a = np - 1; a >= 0; --a) {",
     "for (int a = np - 1; a >= np; --a) {"),
    ("partition.cpp", "RCB cut along the shorter side", "const double* c = (xmax - xmin >= ymax - ymin) ? cx : cy;",
     "const double* c = (xmax - xmin >= ymax - ymin) ? cy : cx;"),
    ("partition.cpp", "RCB halves for odd part counts", "size_t nl = (n * (size_t)kl) / (size_t)k;",
     "size_t nl = n / 2;"),
    ("mesh.cpp", "centroid divisor 2 instead of 3", "m.cx[e] = sx / (3.0 * a2);", "m.cx[e] = sx / (2.0 * a2);"),
    ("util.cpp", "Lanczos diagonal with alpha_j for alpha_{j-1}", "beta[j - 1] / alpha[j - 1]", "beta[j - 1] / alpha[j]"),
    ("util.cpp", "Lanczos off-diagonal without the square root", "e[j] = std::sqrt(beta[j]) / alpha[j];",
     "e[j] = beta[j] / alpha[j];"),
]


def copy_tree(dst):
    for d in (PKG, "include", "oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d),
                        ignore=shutil.ignore_patterns("__pycache__", "_lib", "_build"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)


def build_and_test(cwd):
    b = subprocess.run([sys.executable, "-m", f"{PKG}.build", "--force"], cwd=cwd, capture_output=True, text=True)
    if b.returncode != 0:
        return None, b.stderr[-500:]
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_library_host.py", "-q", "-x", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=cwd, capture_output=True, text=True)
    failed = [line.split(" ")[1] for line in r.stdout.splitlines() if line.startswith("FAILED")]
    return r.returncode, failed


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("-k", default="", help="only mistakes whose file or description contains this text")
    args = ap.parse_args()
    chosen = [m for m in MUTANTS if args.k in m[0] or args.k in m[1]]
    survived = 0
    with tempfile.TemporaryDirectory() as base:
        clean = os.path.join(base, "clean")
        copy_tree(clean)
        rc, failed = build_and_test(clean)
        if rc != 0:
            print(f"the unmodified library fails its host tests: {failed}")
            return 1
        for i, (src, what, old, new) in enumerate(chosen):
            work = os.path.join(base, f"m{i}")
            copy_tree(work)
            path = os.path.join(work, PKG, "csrc", src)
            text = open(path).read()
            if text.count(old) != 1:
                print(f"{what}: the original text occurs {text.count(old)} times in {src}; update this list")
                return 1
            open(path, "w").write(text.replace(old, new))
            t = time.time()
            rc, failed = build_and_test(work)
            if rc is None:
                print(f"{src:14s} {what:48s} does not build: {failed}")
                return 1
            survived += rc == 0
            print(f"{src:14s} {what:48s} {'caught' if rc else 'SURVIVED'} {time.time() - t:6.1f} s  {failed[:1]}",
                  flush=True)
            shutil.rmtree(work)
    print(f"{len(chosen) - survived} of {len(chosen)} planted mistakes caught")
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main())
