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


def test_tensor_core_roofline_arithmetic(monkeypatch):
    """The tensor-core roofline: 2K useful FLOPs per evaluated pair against the
    measured bf16 peak, the epilogue's FP32 operations beside it (3 per pair,
    1.5 for the folded count), and for the folded count the MMA work it
    executes (2 (K + 16) FLOPs per pair) beside the useful work.  (The FP32
    peak needs the GPU's SM count; here it is the GB300's 152 SMs.)"""
    monkeypatch.setattr(bench, "fp32_peak_tops", lambda: (152 * 128 * 2.07e9 / 1e12, 152))
    peaks = bench.load_peaks()
    pairs = [4 * 10 ** 10, 7 * 10 ** 9, 10 ** 10, 0]
    ms = 5.0
    for folded in (False, True):
        r = bench.roofline("tc_count", ms, pairs, 200_000, 64, None, "highd", None, folded)
        assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
        assert math.isclose(r["achieved"], 2 * 64 * pairs[0] / (ms * 1e-3) / 1e12)
        assert math.isclose(r["frac"], r["achieved"] / peaks["bf16_tflops"])
        assert r["epilogue_fp32"]["ops_per_pair"] == (1.5 if folded else 3)
        if folded:
            ex = r["mma_executed"]
            assert ex["flops_per_pair"] == 2 * (64 + 16)
            assert math.isclose(ex["achieved"], r["achieved"] * 80 / 64)
        else:
            assert "mma_executed" not in r
    # other passes keep 3 operations per pair and report no executed MMA rate, folded or not
    r = bench.roofline("tc_union", ms, pairs, 200_000, 64, None, "highd", None, True)
    assert r["epilogue_fp32"]["ops_per_pair"] == 3 and "mma_executed" not in r
    # d = 48 pads to K = 48
    r = bench.roofline("tc_border", ms, pairs, 200_000, 48, None, "highd", None, False)
    assert math.isclose(r["achieved"], 2 * 48 * pairs[2] / (ms * 1e-3) / 1e12)
