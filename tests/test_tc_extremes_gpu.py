"""Tensor-core Gram path at the coordinate extremes, where its exactness argument is tight.

The FP16 form is exact because every centred unit v = u - 512 lies in
[-512, 511], so each product v_p v_q is at most 2^18 and a d = 64 dot product
stays within 2^24 in magnitude, where FP32 holds every integer.  Inputs made of
u in {0, 1, 511, 512, 1022, 1023} drive G = v_p . v_q to +2^24 (two all-zero
points at d = 64) and to -d*512*511 (zero against 1023), and the thresholds
below put T exactly on pair distances that occur in the input and just under
2^24.  Each case forces the FP16 and the two-term BF16 tensor-core passes
(whatever n), checks the diagnostic pass (every pair decided both ways, exact
recheck on the device) and compares counts, core flags and labels with the
oracle, bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1506_02226_gb300 import binding as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EXTREMES = np.array([0, 1, 511, 512, 1022, 1023])


def threshold(eps32: float) -> int:
    """T = floor(eps^2 2^20) for a float32 eps (exact in double: a 48-bit square)."""
    e = float(np.float32(eps32))
    return math.floor(e * e * 1048576.0)


def eps_hitting(D: int):
    """A float32 eps whose threshold is exactly D, or None (consecutive float32
    values near eps move eps^2 2^20 by about 2 eps 2^20 ulp, so not every D is hit)."""
    e = np.float32(math.sqrt(D / 1048576.0))
    for k in range(-6, 7):
        c = e
        step = np.float32(np.inf) if k > 0 else np.float32(-np.inf)
        for _ in range(abs(k)):
            c = np.nextafter(c, step)
        if c > 0 and threshold(float(c)) == D:
            return float(c)
    return None


def extreme_points(seed: int, n: int, d: int) -> np.ndarray:
    """Rows of the grid's extreme units in blocks that push G to its bounds:
    all 0 (v = -512), all 1023 (v = 511), 0/1023 mixtures (opposite signs),
    random picks from EXTREMES, and copies of those with one unit moved by 1
    (pair distances D and D +- small)."""
    rng = np.random.default_rng(seed)
    u = rng.choice(EXTREMES, size=(n, d))
    k = n // 8
    u[:k] = 0
    u[k:2 * k] = 1023
    u[2 * k:3 * k] = np.where(rng.random((k, d)) < 0.5, 0, 1023)
    base = u[3 * k:4 * k].copy()
    moved = base.copy()
    col = rng.integers(0, d, size=k)
    rows = np.arange(k)
    moved[rows, col] = np.where(moved[rows, col] == 0, 1, moved[rows, col] - 1)
    u[4 * k:5 * k] = moved
    u = u[rng.permutation(n)]
    return u.astype(np.float32) / np.float32(1024)


def thresholds_for(u: np.ndarray, rng) -> list:
    """T values on distances the input holds: 0, 1, 1023^2, the smallest,
    median and largest sampled distances below 2^24 - 1 and a few near 2^24,
    plus the largest threshold below 2^24 (eps just under 4)."""
    n, d = u.shape
    a = rng.integers(0, n, size=4000)
    b = rng.integers(0, n, size=4000)
    D = np.unique(((u[a] - u[b]) ** 2).sum(1))
    D = D[(D > 0) & (D < (1 << 24) - 1)]
    picks = [D[0], D[len(D) // 2], D[-1]] if len(D) else []
    picks += [v for v in D[::-1][:40] if v > (1 << 23)][:3]
    # T = 0 (duplicates only), T = 1 (one unit apart) and T = 1023^2, all exact in float32
    out = [1 / 2048, 1 / 1024, 1023 / 1024]
    for v in picks:
        e = eps_hitting(int(v))
        if e is not None and e not in out:
            out.append(e)
    out.append(float(np.nextafter(np.float32(4.0), np.float32(0.0))))  # T = 2^24 - 2
    return out


def run_plan(x, eps, min_pts, prec):
    from paper_1506_02226_gb300.api import Plan
    n, d = x.shape
    with Plan(max_n=n, max_d=d, grid=B.DBSCAN_GRID_OFF, precision=prec) as p:
        lab, cnt, core, st = p.run_detail(torch.from_numpy(x).cuda(), eps, min_pts)
    assert st["path"] == B.DBSCAN_PATH_ALLPAIRS_TC
    return lab.cpu().numpy(), cnt.cpu().numpy(), core.cpu().numpy().astype(bool), st


def verify(x, eps, bf16):
    from paper_1506_02226_gb300.api import Plan
    n, d = x.shape
    xt = torch.from_numpy(x).cuda()
    with Plan(max_n=n, max_d=d) as p:
        return B.dbscan_tc_verify(p.handle, xt.data_ptr(), n, d, eps, bf16)


def test_eps_hitting_gives_the_threshold():
    for D in (1, 2, 260100, 1046529, 16744464, (1 << 24) - 2):
        e = eps_hitting(D)
        assert e is None or threshold(e) == D
    assert threshold(float(np.nextafter(np.float32(4.0), np.float32(0.0)))) == (1 << 24) - 2


@pytest.mark.parametrize("d", [16, 48, 64])
def test_extreme_units_band_and_parity(d):
    n = 4099  # ragged against the 128-row and 256-column tiles
    x = extreme_points(1000 + d, n, d)
    u = np.rint(x.astype(np.float64) * 1024).astype(np.int64)
    v = u - 512
    assert (v == -512).all(1).any() and (v == 511).all(1).any()
    K = -(-d // 16) * 16
    rng = np.random.default_rng(d)
    eps_list = thresholds_for(u, rng)
    assert len(eps_list) >= 3
    for eps in eps_list:
        T = threshold(eps)
        assert T < (1 << 24)
        f16 = verify(x, eps, 0)
        assert f16["pairs"] == n * n and f16["threshold"] == min(T, d * 1023 * 1023)
        assert f16["wrong_outside_band"] == 0, (d, T, f16)
        assert f16["max_abs_error_2g"] == 0, (d, T, f16)
        b16 = verify(x, eps, 1)
        assert b16["wrong_outside_band"] == 0, (d, T, b16)
        assert b16["max_abs_error_2g"] <= 14 * K, (d, T, b16)
        for min_pts in (2, 40):
            want_lab, want_cnt, want_core = oracle.dbscan(x, eps, min_pts)
            for prec in (B.DBSCAN_PREC_FP16_GRAM, B.DBSCAN_PREC_BF16_GRAM):
                lab, cnt, core, _ = run_plan(x, eps, min_pts, prec)
                np.testing.assert_array_equal(cnt, want_cnt, err_msg=f"d={d} T={T} prec={prec}")
                np.testing.assert_array_equal(core, want_core, err_msg=f"d={d} T={T} prec={prec}")
                np.testing.assert_array_equal(lab, want_lab, err_msg=f"d={d} T={T} prec={prec} mp={min_pts}")


@pytest.mark.parametrize("unit", [0, 1023])
def test_identical_points_at_the_ends(unit):
    """Every point the same (G = 2^24 for unit 0 at d = 64): all mutual
    neighbours at any eps, one cluster with id 0."""
    n, d = 4096, 64
    x = np.full((n, d), np.float32(unit / 1024), dtype=np.float32)
    for eps in (1 / 2048, float(np.nextafter(np.float32(4.0), np.float32(0.0)))):
        for bf16 in (0, 1):
            rep = verify(x, eps, bf16)
            assert rep["wrong_outside_band"] == 0
            if not bf16:
                assert rep["max_abs_error_2g"] == 0
        for prec in (B.DBSCAN_PREC_FP16_GRAM, B.DBSCAN_PREC_BF16_GRAM):
            lab, cnt, core, st = run_plan(x, eps, 5, prec)
            assert (cnt == n).all() and core.all() and (lab == 0).all()
            assert st["n_clusters"] == 1


# Largest max |v|^2 for which the FP16 count folds the column norm into the
# MMA: its accumulator G - ceil(|v_q|^2 / 2) is exact while
# 3 max|v|^2 + 1 <= 2^25 (every partial sum then stays within 2^24).
FOLD_LIMIT = ((1 << 25) - 1) // 3


def fold_edge_points(seed: int, n: int, d: int, over: bool) -> np.ndarray:
    """Rows whose largest |v|^2 sits just below (over=False) or just above
    (over=True) the folded count's limit: 42 coordinates at the grid's ends
    (v = -512 or 511) and one at +-418 (or +-419), so that G reaches about
    +-1.1e7 between aligned and opposite rows; sign flips of shared base rows
    put pair distances at every multiple of about 1023^2 below 2^24; copies
    with one coordinate moved by one unit give distances next to those; the
    other rows lie near the centre.  |v|^2 takes both parities."""
    rng = np.random.default_rng(seed)
    k, last = 42, (419 if over else 418)
    v = rng.integers(-40, 41, size=(n, d))
    m = (3 * n) // 4
    base = rng.choice([-512, 511], size=(64, k))
    rows = base[rng.integers(0, 64, size=m)].copy()
    for i in range(m):
        j = rng.integers(0, 16)
        c = rng.choice(k, size=j, replace=False)
        rows[i, c] = np.where(rows[i, c] == -512, 511, -512)
    v[:m] = 0
    v[:m, :k] = rows
    v[:m, k] = rng.choice([-last, last], size=m)
    v[0, :k] = -512  # the largest norm of the set
    near = rng.integers(1, m, size=m // 4)
    col = rng.integers(0, k + 1, size=near.size)
    v[near, col] -= np.sign(v[near, col])
    beta = (v.astype(np.int64) ** 2).sum(1)
    assert (beta.max() > FOLD_LIMIT) == over and (beta & 1).any() and not (beta & 1).all()
    u = v[rng.permutation(n)] + 512
    return u.astype(np.float32) / np.float32(1024)


@pytest.mark.parametrize("over", [False, True])
def test_folded_count_at_its_norm_limit(over):
    """The FP16 count runs its folded form up to the norm limit and falls back
    to G alone above it; both give the oracle's exact counts, cores and labels."""
    from paper_1506_02226_gb300.api import Plan
    n, d = 4099, 64
    x = fold_edge_points(2000 + int(over), n, d, over)
    u = np.rint(x.astype(np.float64) * 1024).astype(np.int64)
    rng = np.random.default_rng(5 + int(over))
    for eps in thresholds_for(u, rng):
        T = threshold(eps)
        for min_pts in (2, 40):
            want_lab, want_cnt, want_core = oracle.dbscan(x, eps, min_pts)
            with Plan(max_n=n, max_d=d, grid=B.DBSCAN_GRID_OFF, precision=B.DBSCAN_PREC_FP16_GRAM) as p:
                lab, cnt, core, st = p.run_detail(torch.from_numpy(x).cuda(), eps, min_pts)
                folded = p.counters()[15]
            assert st["path"] == B.DBSCAN_PATH_ALLPAIRS_TC
            assert folded == (0 if over else 1), (T, folded)
            np.testing.assert_array_equal(cnt.cpu().numpy(), want_cnt, err_msg=f"T={T} over={over}")
            np.testing.assert_array_equal(core.cpu().numpy().astype(bool), want_core)
            np.testing.assert_array_equal(lab.cpu().numpy(), want_lab, err_msg=f"T={T} mp={min_pts} over={over}")
