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
