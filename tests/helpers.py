"""Shared test fixtures: seeded problems built from the synthetic input generators."""
from __future__ import annotations

import functools

import numpy as np

from synth.voronoi import voronoi_mesh


def f_sin(X):
    return 2 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])


def u_sin(X):
    return np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])


@functools.lru_cache(maxsize=16)
def mesh(n, seed, lloyd=20):
    return voronoi_mesh(n, seed, lloyd=lloyd)


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def paper_table(example: int, p: int):
    """The paper's printed K(P_ad) and iteration counts (Sec. 7, Example 2 or 4, p = q), from the cited
    fixture tests/golden/paper_example{example}_p{p}.txt: {(N_h, N_H): (K, iterations)}."""
    out = {}
    with open(f"{GOLDEN}/paper_example{example}_p{p}.txt") as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            nh, nH, K, it = line.split()
            out[(int(nh), int(nH))] = (float(K), int(it))
    return out
