"""The projected grid for 4 <= d <= 8 against the oracle, bit for bit.

Cells are keyed on the first three coordinates with side floor(sqrt(T)) + 1
units, so every neighbour lies in the 27 surrounding cells of the projection;
each candidate pair is then decided exactly over all d coordinates.  Counts,
core flags and labels (both label modes) must equal the oracle's on ragged
sizes (around the 32-point chunks), dense cells (every point in one cell),
thresholds on and next to pair distances, the degenerate cases, and the
200,000-point workload at d = 4 and d = 8.
"""
import numpy as np
import pytest

import oracle
from paper_1506_02226_gb300 import binding as B
from paper_1506_02226_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(points, eps, min_pts, grid=B.DBSCAN_GRID_ON, label_mode=0, exact=True, max_n=None):
    from paper_1506_02226_gb300.api import Plan
    n, d = points.shape
    x = torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).cuda()
    with Plan(max_n=max(n, 1, max_n or 0), max_d=d, grid=grid, label_mode=label_mode) as p:
        if exact:
            lab, cnt, core, st = p.run_detail(x, eps, min_pts)
            return lab.cpu().numpy(), cnt.cpu().numpy(), core.cpu().numpy().astype(bool), st, p.pair_tests()
        lab, st = p.run(x, eps, min_pts, stats=True)
        return lab.cpu().numpy(), None, None, st, p.pair_tests()


def check(points, eps, min_pts, modes=(0, 1)):
    for mode in modes:
        want_lab, want_cnt, want_core = oracle.dbscan(points, eps, min_pts, label_mode=mode)
        lab, cnt, core, st, ev = run(points, eps, min_pts, label_mode=mode)
        assert st["path"] == B.DBSCAN_PATH_GRID_PROJECTED
        np.testing.assert_array_equal(cnt, want_cnt)
        np.testing.assert_array_equal(core, want_core)
        np.testing.assert_array_equal(lab, want_lab, err_msg=f"mode={mode}")
        assert st["n_core"] == int(want_core.sum())
        assert st["n_core"] + st["n_border"] + st["n_noise"] == points.shape[0]
        n = points.shape[0]
        assert st["candidate_pairs"] >= int(want_cnt.sum())  # every neighbour pair is a candidate
        assert ev[0] <= st["candidate_pairs"] and st["pair_tests"] == sum(ev)
        lab2, _, _, _, _ = run(points, eps, min_pts, label_mode=mode, exact=False)  # early exit, as timed
        np.testing.assert_array_equal(lab2, want_lab)


def blobs(seed, n, d, spread):
    rng = np.random.default_rng(seed)
    centres = rng.integers(60, 960, size=(7, d))
    u = np.clip(centres[rng.integers(0, 7, size=n)] + rng.integers(-spread, spread + 1, size=(n, d)), 0, 1023)
    noise = rng.random(n) < 0.15
    u[noise] = rng.integers(0, 1024, size=(int(noise.sum()), d))
    return u.astype(np.float32) / np.float32(1024)


@pytest.mark.parametrize("d", [4, 5, 7, 8])
@pytest.mark.parametrize("n", [1, 2, 31, 33, 1000, 4099])
def test_ragged(n, d):
    x = blobs(10 * n + d, n, d, spread=12)
    check(x, float(np.float32(14 * np.sqrt(d) / 1024)), 4)


@pytest.mark.parametrize("d", [4, 8])
def test_dense_cells_span_many_chunks(d):
    """Thousands of points in a few cells (chunks of 32 from one cell on many warps)."""
    rng = np.random.default_rng(d)
    u = np.concatenate([np.full((3000, d), 500), 500 + rng.integers(-3, 4, size=(2000, d)),
                        rng.integers(0, 1024, size=(500, d))])
    x = (u.astype(np.float32) / np.float32(1024))[rng.permutation(5500)]
    for eps, mp in ((4 / 1024, 10), (0.5 / 1024, 2), (20 / 1024, 3000)):
        check(x, eps, mp, modes=(0,))


def test_thresholds_on_pair_distances():
    rng = np.random.default_rng(5)
    for d in (4, 6, 8):
        u = np.clip(300 + rng.integers(-40, 41, size=(3000, d)), 0, 1023)
        x = u.astype(np.float32) / np.float32(1024)
        D = ((u[0] - u[1:]) ** 2).sum(1)
        for q in (0.05, 0.3, 2):
            eps = float(np.sqrt(np.percentile(D, q)) / 1024)  # float32 rounding lands T near a real D
            check(x, eps, 8, modes=(0,))


def test_degenerate_and_fallback():
    rng = np.random.default_rng(9)
    x = (rng.integers(0, 200, size=(3000, 5)).astype(np.float32) / np.float32(1024))
    check(x, 0.5 / 1024, 2, modes=(0,))  # T = 0: only duplicates are neighbours
    check(x, 8 / 1024, 1, modes=(0,))  # min_pts = 1: components of the eps-graph
    check(x, 8 / 1024, 3001, modes=(0,))  # min_pts > n: all noise
    dup = np.full((700, 6), np.float32(0.25), dtype=np.float32)
    check(dup, 1e-3, 5, modes=(0, 1))  # every point identical, one cell
    # eps too large for cells to prune (fewer than 4 per axis): AUTO falls back to
    # all pairs, ON reports it unsupported
    lab, _, _, st, _ = run(x, 0.4, 5, grid=B.DBSCAN_GRID_AUTO)
    assert st["path"] == B.DBSCAN_PATH_ALLPAIRS_SIMT
    np.testing.assert_array_equal(lab, oracle.dbscan(x, 0.4, 5)[0])
    from paper_1506_02226_gb300.api import Plan
    with Plan(max_n=3000, max_d=5, grid=B.DBSCAN_GRID_ON) as p:
        lab = torch.empty(3000, dtype=torch.int32, device="cuda")
        xt = torch.from_numpy(x).cuda()
        assert B.dbscan_run(p.handle, xt.data_ptr(), 3000, 5, 0.4, 5, lab.data_ptr()) == B.DBSCAN_ERR_UNSUPPORTED
        bad = xt.clone()
        bad[17, 4] = 0.3  # off the grid in a coordinate the cells do not use
        assert B.dbscan_run(p.handle, bad.data_ptr(), 3000, 5, 8 / 1024, 5, lab.data_ptr()) == \
            B.DBSCAN_ERR_NOT_QUANTISED


def test_auto_takes_the_projected_grid():
    inst = inputs.mid_d(6, n=30_000)
    lab, _, _, st, ev = run(inst.points, inst.eps, inst.min_pts, grid=B.DBSCAN_GRID_AUTO, exact=False)
    assert st["path"] == B.DBSCAN_PATH_GRID_PROJECTED
    assert 0 < st["pair_tests"] < inst.n ** 2 / 10
    np.testing.assert_array_equal(lab, oracle.dbscan(inst.points, inst.eps, inst.min_pts)[0])


@pytest.mark.slow
@pytest.mark.parametrize("d", [4, 8])
def test_full_size_mid_d_workload(d):
    """n = 200,000 on the projected grid, as bench.py runs it, against the full oracle."""
    inst = inputs.mid_d(d)
    want_lab, want_cnt, want_core = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
    lab, cnt, core, st, _ = run(inst.points, inst.eps, inst.min_pts, grid=B.DBSCAN_GRID_AUTO)
    assert st["path"] == B.DBSCAN_PATH_GRID_PROJECTED
    np.testing.assert_array_equal(cnt, want_cnt)
    np.testing.assert_array_equal(core, want_core)
    np.testing.assert_array_equal(lab, want_lab)
    lab2, _, _, _, _ = run(inst.points, inst.eps, inst.min_pts, grid=B.DBSCAN_GRID_AUTO, exact=False)
    np.testing.assert_array_equal(lab2, want_lab)
