"""Seeded problem mixes for the batching and serving workloads (inputs only).

A problem is (element count, degree, mesh seed, coefficient seed).  Element counts are log-uniform in
[1024, 16384], degrees uniform in {1, 2, 3, 4}; the solver side uses N/256 subdomains and N/64 coarse
agglomerates at p_c = 1, and one diffusion coefficient per subdomain, log-uniform in [1, 1e3].
Meshes are built in worker processes started with the spawn method (safe before or after a GPU context).
"""
from __future__ import annotations

from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp
import os

import numpy as np

from .voronoi import PolyMesh, voronoi_mesh


def problem_specs(count: int, seed: int, lo: int = 1024, hi: int = 16384):
    """count problems drawn from numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(2.0 ** rng.uniform(np.log2(lo), np.log2(hi))))
        p = int(rng.integers(1, 5))
        out.append({"index": i, "n_elem": n, "p": p, "mesh_seed": int(rng.integers(1, 2 ** 31 - 1)),
                    "coef_seed": int(rng.integers(1, 2 ** 31 - 1)), "nsub": max(1, n // 256),
                    "ncoarse": max(1, n // 64)})
    return out


def _mesh(args) -> PolyMesh:
    n, seed = args
    return voronoi_mesh(n, seed)


def build_meshes(specs, workers: int | None = None):
    """Voronoi meshes of every spec, built in parallel (spawned workers)."""
    jobs = [(s["n_elem"], s["mesh_seed"]) for s in specs]
    workers = workers or max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    if workers == 1:
        return [_mesh(j) for j in jobs]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_mesh, jobs))
