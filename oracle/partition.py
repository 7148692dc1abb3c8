"""Subdomain partition T_H (Sec. 3) and coarse agglomerates T_H (nested case, Remark 3.1).

The paper builds both partitions by agglomerating fine elements (Sec. 7, Example 2; Metis in
Example 1) and fixes no algorithm.  Reading adopted: recursive coordinate bisection (RCB) of the
element area centroids.  A set of elements is split into k parts by cutting along the longer side
of its centroid bounding box (x when the extents tie), after sorting by (coordinate, element
index); the first floor(k/2) parts receive floor(n * floor(k/2) / k) elements.  Parts are numbered
in depth-first, lower-side-first order.

Coarse agglomerates: when ncoarse >= nsub, subdomain i is split by RCB into
c_i = floor((i+1) nc / ns) - floor(i nc / ns) agglomerates (numbered subdomain by subdomain), so
the agglomerates are nested in both the fine mesh and the subdomains; when ncoarse < nsub the
agglomerates are an RCB of the whole mesh into ncoarse parts.
"""
from __future__ import annotations

import numpy as np


def rcb(points: np.ndarray, elems: np.ndarray, k: int):
    """Split ``elems`` (indices into ``points``) into k parts; returns a list of index arrays."""
    elems = np.asarray(elems)
    if k <= 1:
        return [elems]
    xs = points[elems, 0]
    ys = points[elems, 1]
    ext_x = xs.max() - xs.min()
    ext_y = ys.max() - ys.min()
    coord = xs if ext_x >= ext_y else ys
    order = np.lexsort((elems, coord))
    sorted_elems = elems[order]
    kl = k // 2
    nl = (len(elems) * kl) // k
    return rcb(points, sorted_elems[:nl], kl) + rcb(points, sorted_elems[nl:], k - kl)


def subdomains(centroids: np.ndarray, nsub: int) -> np.ndarray:
    ne = len(centroids)
    parts = rcb(centroids, np.arange(ne), nsub)
    sub = np.empty(ne, dtype=np.int32)
    for i, part in enumerate(parts):
        sub[part] = i
    return sub


def agglomerates(centroids: np.ndarray, sub: np.ndarray, nsub: int, ncoarse: int) -> np.ndarray:
    ne = len(centroids)
    agg = np.empty(ne, dtype=np.int32)
    if ncoarse >= nsub:
        nxt = 0
        for i in range(nsub):
            ci = (i + 1) * ncoarse // nsub - i * ncoarse // nsub
            members = np.nonzero(sub == i)[0]
            for part in rcb(centroids, members, ci):
                agg[part] = nxt
                nxt += 1
    else:
        for j, part in enumerate(rcb(centroids, np.arange(ne), ncoarse)):
            agg[part] = j
    return agg


def subdomain_adjacency(sub: np.ndarray, faces) -> list:
    ns = int(sub.max()) + 1
    adj = [set() for _ in range(ns)]
    for (ep, em, _, _) in faces:
        if em >= 0 and sub[ep] != sub[em]:
            adj[sub[ep]].add(int(sub[em]))
            adj[sub[em]].add(int(sub[ep]))
    return adj


def greedy_colouring(adj: list) -> np.ndarray:
    """Colour subdomains so that neighbours (shared boundary) differ; the number of colours bounds
    how many A-orthogonal groups the local projections fall into (Sec. 5, Lemma decVi)."""
    col = -np.ones(len(adj), dtype=int)
    for i in range(len(adj)):
        used = {col[j] for j in adj[i] if col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return col
