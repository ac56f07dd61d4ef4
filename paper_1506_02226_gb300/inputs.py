"""Seeded synthetic inputs for the exact DBSCAN path (input generation only).

This module draws points and per-instance parameters. It holds none of the
clustering arithmetic: no neighbour predicate, no core test, no merging. Both
the CUDA path (through ``bench.py`` and the GPU tests) and the CPU oracle (in
the tests) take their inputs from here, so neither side generates data for the
other.

Every coordinate lies on the 2^-10 grid in [0, 1): ``x = u / 1024`` with
integer ``u`` in 0..1023. Points are row-major ``float32[n, d]``.

The paper evaluates on one unnamed 3-D point set of 5061, 23040 and 60032
points (Section V, Table V) that is not available; these seeded blob-plus-noise
mixtures stand in for it. The recipe readings (how Gaussian samples outside
[0, 1) are handled, how blob sizes are split, the per-dimension sigma of the
batched and served mixtures) are spelled out on each function.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GRID = 1024  # coordinates are multiples of 2^-10
SEED_BASE = 150602226


@dataclasses.dataclass(frozen=True)
class Instance:
    """One clustering problem: points plus its eps and min_pts."""

    points: np.ndarray  # float32 [n, d], row-major, on the 2^-10 grid
    eps: float  # float32 value, stored as a Python float
    min_pts: int

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def d(self) -> int:
        return int(self.points.shape[1])


def _resample_unit(rng: np.random.Generator, centre: np.ndarray, sigma: float, m: int) -> np.ndarray:
    """Gaussian samples around ``centre``; every coordinate outside [0, 1) is
    redrawn until it falls inside (clamping would pile duplicates on the faces)."""
    d = centre.shape[0]
    x = centre[None, :] + sigma * rng.standard_normal((m, d))
    bad = (x < 0.0) | (x >= 1.0)
    while bad.any():
        rows, cols = np.nonzero(bad)
        x[rows, cols] = centre[cols] + sigma * rng.standard_normal(rows.shape[0])
        bad = (x < 0.0) | (x >= 1.0)
    return x


def blobs_plus_noise(rng: np.random.Generator, n: int, d: int, sigmas, noise_frac: float) -> np.ndarray:
    """``len(sigmas)`` isotropic Gaussian blobs with uniform centres, plus uniform noise.

    ``round(noise_frac * n)`` points are uniform in [0,1)^d. The rest are split
    equally over the blobs, the remainder going to the lowest-index blobs. The
    rows are then put in a random order, so that a point's index says nothing
    about where it lies. Quantisation is ``u = floor(1024 x)``.
    """
    sigmas = [float(s) for s in sigmas]
    k = len(sigmas)
    n_noise = int(round(noise_frac * n)) if k > 0 else n
    n_blob = n - n_noise
    parts = []
    if k > 0 and n_blob > 0:
        centres = rng.random((k, d))
        base, rem = divmod(n_blob, k)
        for b in range(k):
            m = base + (1 if b < rem else 0)
            if m:
                parts.append(_resample_unit(rng, centres[b], sigmas[b], m))
    if n_noise:
        parts.append(rng.random((n_noise, d)))
    x = np.concatenate(parts, axis=0) if parts else np.zeros((0, d))
    x = x[rng.permutation(x.shape[0])]
    u = np.floor(x * GRID).astype(np.int64)
    np.clip(u, 0, GRID - 1, out=u)  # x < 1 already; guards float rounding at the top edge
    return (u.astype(np.float32) / np.float32(GRID)).astype(np.float32)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def small_2d(seed: int = SEED_BASE + 1) -> Instance:
    """n=2000, d=2: 90% from 5 Gaussians (sigma 0.03), 10% noise; eps 0.02, min_pts 5."""
    rng = np.random.default_rng(seed)
    pts = blobs_plus_noise(rng, 2000, 2, [0.03] * 5, 0.10)
    return Instance(pts, float(np.float32(0.02)), 5)


def large_lowd(d: int = 2, n: int = 500_000, seed: int | None = None) -> Instance:
    """n=500,000, d=2 or 3: 50 blobs, sigma log-uniform in [0.002, 0.02], 20% noise;
    eps 0.005, min_pts 10. ``n`` may be lowered for a subsample of the same recipe."""
    if seed is None:
        seed = SEED_BASE + 2 + (0 if d == 2 else 100)
    rng = np.random.default_rng(seed)
    sig = np.exp(rng.uniform(math.log(0.002), math.log(0.02), size=50))
    pts = blobs_plus_noise(rng, n, d, sig, 0.20)
    return Instance(pts, float(np.float32(0.005)), 10)


def mid_d(d: int = 8, n: int = 200_000, seed: int | None = None) -> Instance:
    """4 <= d <= 8 (the projected-grid path): the d <= 3 recipe's 50 blobs, sigma
    log-uniform in [0.002, 0.02] per coordinate, 20% noise, with eps scaled to
    the dimension, 0.005 * sqrt(d / 2) (the typical distance of two points of a
    blob grows as sqrt(d)), min_pts 10."""
    if not 4 <= d <= 8:
        raise ValueError("mid_d is the 4 <= d <= 8 recipe")
    if seed is None:
        seed = SEED_BASE + 6 + 100 * d
    rng = np.random.default_rng(seed)
    sig = np.exp(rng.uniform(math.log(0.002), math.log(0.02), size=50))
    pts = blobs_plus_noise(rng, n, d, sig, 0.20)
    return Instance(pts, float(np.float32(0.005 * math.sqrt(d / 2))), 10)


def paper_3d(n: int = 23_040, seed: int = SEED_BASE + 7) -> Instance:
    """A stand-in for the paper's unnamed 3-D point set at its middle size
    (N = 23,040, Section V): the d <= 3 recipe (50 blobs, sigma log-uniform in
    [0.002, 0.02], 20% noise) with eps 0.02 and min_pts 10 (the paper gives
    neither)."""
    rng = np.random.default_rng(seed)
    sig = np.exp(rng.uniform(math.log(0.002), math.log(0.02), size=50))
    return Instance(blobs_plus_noise(rng, n, 3, sig, 0.20), float(np.float32(0.02)), 10)


# eps of the d=64 workload: the median over 2,000 seeded query points of the
# distance to the 30th nearest point (the query itself counted), rounded to
# float32.  Written by ``derive_highd_eps()`` below and frozen here.
HIGHD_EPS = 0.4566502869129181
HIGHD_QUERIES = 2000
HIGHD_K = 30


def _highd_points(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return blobs_plus_noise(rng, n, 64, [0.05] * 100, 0.15)


def high_d(n: int = 200_000, seed: int = SEED_BASE + 3, eps: float | None = None) -> Instance:
    """n=200,000, d=64: 100 blobs (sigma 0.05 per dimension), 15% noise; min_pts 20;
    eps frozen in ``HIGHD_EPS`` (median 30-NN distance)."""
    pts = _highd_points(n, seed)
    return Instance(pts, float(np.float32(HIGHD_EPS if eps is None else eps)), 20)


def derive_highd_eps(n: int = 200_000, seed: int = SEED_BASE + 3) -> float:
    """Recompute the frozen eps of ``high_d``: median 30-NN distance of 2000 queries.

    Squared distances are formed in float64 from the integer grid units, which is
    exact here (every partial sum is an integer below 2^53).
    """
    pts = _highd_points(n, seed)
    u = np.rint(pts.astype(np.float64) * GRID)
    rng = np.random.default_rng(seed + 7)
    q = rng.choice(n, size=HIGHD_QUERIES, replace=False)
    nrm = (u * u).sum(axis=1)
    kth = np.empty(HIGHD_QUERIES)
    for s in range(0, HIGHD_QUERIES, 100):
        qi = q[s:s + 100]
        dd = nrm[qi][:, None] + nrm[None, :] - 2.0 * (u[qi] @ u.T)
        kth[s:s + 100] = np.partition(dd, HIGHD_K - 1, axis=1)[:, HIGHD_K - 1]
    med = float(np.median(kth))
    return float(np.float32(math.sqrt(med) / GRID))


def _mixture_instance(rng: np.random.Generator, n: int, d: int) -> Instance:
    """One instance of the batched/served recipe: 1-8 blobs plus 10% noise.

    Reading: per-blob sigma is log-uniform in [0.005, 0.03] scaled by sqrt(2/d),
    so that the typical distance between two points of one blob (sigma*sqrt(2d))
    is 0.01-0.06 at every d, the same range as eps in [0.01, 0.05].
    """
    k = int(rng.integers(1, 9))
    sig = np.exp(rng.uniform(math.log(0.005), math.log(0.03), size=k)) * math.sqrt(2.0 / d)
    pts = blobs_plus_noise(rng, n, d, sig, 0.10)
    eps = float(np.float32(rng.uniform(0.01, 0.05)))
    min_pts = int(rng.integers(4, 17))
    return Instance(pts, eps, min_pts)


def batch_sizes(count: int = 4096, seed: int = SEED_BASE + 4):
    """(n, d) of each batched instance: n log-uniform in [64, 8192], d in {2, 3, 16}."""
    rng = np.random.default_rng(seed)
    n = np.floor(np.exp(rng.uniform(math.log(64), math.log(8192), size=count))).astype(np.int64)
    d = rng.choice(np.array([2, 3, 16]), size=count)
    return n, d


def batch(count: int = 4096, seed: int = SEED_BASE + 4) -> list[Instance]:
    """The batched workload: ``count`` independent instances (default 4,096)."""
    ns, ds = batch_sizes(count, seed)
    out = []
    for i in range(count):
        rng = np.random.default_rng([seed, i])
        out.append(_mixture_instance(rng, int(ns[i]), int(ds[i])))
    return out


def serve_job(i: int, seed: int = SEED_BASE + 5, n_max: int = 500_000) -> Instance:
    """Job ``i`` of the served workload: n log-uniform in [1000, n_max], d in {2, 3, 32}."""
    rng = np.random.default_rng([seed, i])
    n = int(math.floor(math.exp(rng.uniform(math.log(1000), math.log(n_max)))))
    d = int(rng.choice(np.array([2, 3, 32])))
    return _mixture_instance(rng, n, d)


def serve_arrivals(count: int, rate_per_s: float, seed: int = SEED_BASE + 5) -> np.ndarray:
    """Poisson arrival times (seconds from start) of ``count`` jobs at ``rate_per_s``."""
    rng = np.random.default_rng([seed, 1 << 30])
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def subsample(inst: Instance, m: int, seed: int = 0) -> Instance:
    """``m`` rows of ``inst`` chosen uniformly without replacement, same eps/min_pts."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(inst.n, size=m, replace=False))
    return Instance(np.ascontiguousarray(inst.points[idx]), inst.eps, inst.min_pts)
