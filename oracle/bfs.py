"""Second, independent DBSCAN for cross-checking the oracle — TEST INFRASTRUCTURE ONLY.

Classic expand-cluster DBSCAN (the breadth-first search that Section III
attributes to G-DBSCAN), written separately from ``dbscan_oracle.c``:

* It works on the real coordinates in float64, not on integer grid units.  For
  points on the 2^-10 grid every difference, square and sum is exact in
  float64, and eps^2 of a float32 eps is exact too, so ``dist^2 <= eps^2`` is
  decided exactly (Section II, definition 1, with Section IV-B's ``<=``).
* Core points have at least ``min_pts`` neighbours, self included (Section II,
  definition 2).
* Clusters grow by BFS from each unvisited core point in index order
  (definition 3 and the cluster definition of Section II).

It returns both the classic result (a border point keeps the first cluster
that reaches it) and the canonical one (cluster id = smallest core index; a
border point takes the cluster of its smallest-index core neighbour).  Meant
for n up to a few thousand.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def neighbour_lists(points: np.ndarray, eps: float) -> list[np.ndarray]:
    x = np.asarray(points, dtype=np.float64)
    e2 = float(np.float32(eps)) ** 2
    out = []
    for i in range(x.shape[0]):
        diff = x - x[i]
        out.append(np.nonzero((diff * diff).sum(axis=1) <= e2)[0])
    return out


def dbscan_bfs(points: np.ndarray, eps: float, min_pts: int):
    """Returns (classic_labels, canonical_labels, core) as numpy arrays."""
    n = points.shape[0]
    nb = neighbour_lists(points, eps)
    core = np.array([len(l) >= min_pts for l in nb], dtype=bool)
    UNSEEN = -2
    lab = np.full(n, UNSEEN, dtype=np.int64)
    cid = 0
    for i in range(n):
        if lab[i] != UNSEEN:
            continue
        if not core[i]:
            lab[i] = -1  # tentatively noise; a later cluster may claim it
            continue
        lab[i] = cid
        queue = deque([i])
        while queue:
            p = queue.popleft()
            for q in nb[p]:
                if lab[q] == -1:
                    lab[q] = cid  # noise becomes a border point of this cluster
                elif lab[q] == UNSEEN:
                    lab[q] = cid
                    if core[q]:
                        queue.append(q)
        cid += 1
    # Canonical ids: smallest core index of each classic cluster.
    root_of = {}
    for p in range(n):
        if core[p] and lab[p] not in root_of:
            root_of[lab[p]] = p
    classic = np.array([root_of[l] if l >= 0 else -1 for l in lab], dtype=np.int32)
    canon = classic.copy()
    for p in range(n):
        if not core[p]:
            cn = [q for q in nb[p] if core[q]]
            canon[p] = classic[min(cn)] if cn else -1
    return classic, canon, core
