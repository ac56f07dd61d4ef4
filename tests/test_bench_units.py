"""The bench's work units, recounted by brute force on small inputs.

`bench.grid_structure` counts the ordered candidate pairs of the eps-grid (the
pair tests of the G pair-tests/s metric) and the neighbour-list entries (the
algorithmic bytes of the grid kernels).  Here every pair of points and every
pair of occupied cells is enumerated directly.
"""
import itertools
import math

import numpy as np
import pytest

import bench


def _brute(points, eps):
    u = np.rint(points.astype(np.float64) * 1024).astype(np.int64)
    n, d = u.shape
    e = float(np.float32(eps))
    T = min(math.floor(e * e * 1048576.0), d * 1023 * 1023)
    c = math.isqrt(T // d) + 1
    r = -(-math.isqrt(T) // c)
    kept = {o for o in itertools.product(range(-r, r + 1), repeat=d)
            if sum(((abs(x) - 1) * c + 1) ** 2 for x in o if x) <= T}  # includes the zero offset
    cells = [tuple(v) for v in (u // c)]
    pairs = sum(1 for p in range(n) for q in range(n)
                if tuple(a - b for a, b in zip(cells[q], cells[p])) in kept)
    occ = sorted(set(cells))
    near = far = 0
    for a in occ:
        for b in occ:
            o = tuple(x - y for x, y in zip(b, a))
            if any(o) and o in kept:
                if max(abs(x) for x in o) <= 1:
                    near += 1
                else:
                    far += 1
    return pairs, len(occ), near, far


@pytest.mark.parametrize("d,eps", [(1, 7 / 1024), (2, 5 / 1024), (2, 12 / 1024), (3, 6 / 1024)])
def test_grid_structure_matches_brute_force(d, eps):
    rng = np.random.default_rng(40 + d)
    centres = rng.integers(40, 984, size=(4, d))
    u = np.concatenate([centres[rng.integers(0, 4, 250)] + rng.integers(-25, 26, size=(250, d)),
                        rng.integers(0, 1024, size=(50, d))])
    x = (np.clip(u, 0, 1023).astype(np.float32) / np.float32(1024))
    gs = bench.grid_structure(x, eps)
    pairs, cells, near, far = _brute(x, eps)
    assert gs["candidate_pairs"] == pairs
    assert gs["cells"] == cells
    assert (gs["near_entries"], gs["far_entries"]) == (near, far)


def test_candidate_pairs_bound_the_neighbour_pairs():
    """Every eps-neighbour pair is a candidate (the grid misses no pair)."""
    rng = np.random.default_rng(7)
    u = rng.integers(0, 1024, size=(400, 2))
    x = u.astype(np.float32) / np.float32(1024)
    eps = 20 / 1024
    T = math.floor(float(np.float32(eps)) ** 2 * 1048576.0)
    diff = u[:, None, :] - u[None, :, :]
    nbr = (diff ** 2).sum(-1) <= T
    gs = bench.grid_structure(x, eps)
    assert gs["candidate_pairs"] >= int(nbr.sum())
