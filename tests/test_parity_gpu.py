"""CUDA path vs the CPU oracle, bit-exact, through the C ABI.

Labels, neighbour counts and core flags are integers decided by an exact
integer predicate, so the bar is equality.  Covers both candidate paths (the
eps-grid for d <= 3 and all pairs), both label modes, ragged tiles (n around
multiples of the 64-point tile), every exact-arithmetic mode of the all-pairs
kernel (FP32 Gram d <= 8, FP32 direct, INT32 direct), the degenerate cases
(T = 0, eps beyond the diameter, min_pts = 1, min_pts > n, n = 0 and 1,
duplicates), error reporting, the host-buffer entry point, and the full-size
2-D and 3-D workloads.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1506_02226_gb300 import binding as B
from paper_1506_02226_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def gpu_detail(points, eps, min_pts, grid=B.DBSCAN_GRID_AUTO, label_mode=0, precision=B.DBSCAN_PREC_AUTO,
               max_n=None):
    from paper_1506_02226_gb300.api import Plan
    n, d = points.shape
    x = torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).cuda()
    with Plan(max_n=max(n, 1, max_n or 0), max_d=max(d, 1), grid=grid, label_mode=label_mode,
              precision=precision) as p:
        lab, cnt, core, st = p.run_detail(x, eps, min_pts)
    return lab.cpu().numpy(), cnt.cpu().numpy(), core.cpu().numpy().astype(bool), st


def gpu_labels(points, eps, min_pts, grid=B.DBSCAN_GRID_AUTO, label_mode=0):
    from paper_1506_02226_gb300.api import Plan
    n, d = points.shape
    x = torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).cuda()
    with Plan(max_n=max(n, 1), max_d=d, grid=grid, label_mode=label_mode) as p:
        lab, st = p.run(x, eps, min_pts, stats=True)
    return lab.cpu().numpy(), st


def grids_for(d):
    return (B.DBSCAN_GRID_ON, B.DBSCAN_GRID_OFF) if d <= 3 else (B.DBSCAN_GRID_OFF,)


def assert_matches_oracle(points, eps, min_pts, grids=None):
    d = points.shape[1]
    for mode in (0, 1):
        want_lab, want_cnt, want_core = oracle.dbscan(points, eps, min_pts, label_mode=mode)
        for g in (grids or grids_for(d)):
            lab, cnt, core, st = gpu_detail(points, eps, min_pts, grid=g, label_mode=mode)
            np.testing.assert_array_equal(cnt, want_cnt, err_msg=f"counts grid={g}")
            np.testing.assert_array_equal(core, want_core, err_msg=f"core grid={g}")
            np.testing.assert_array_equal(lab, want_lab, err_msg=f"labels grid={g} mode={mode}")
            n = points.shape[0]
            assert st["n_core"] + st["n_border"] + st["n_noise"] == n
            assert st["n_core"] == int(want_core.sum())
            assert st["n_clusters"] == len(set(want_lab[want_lab >= 0].tolist()))


def test_grid_occupancy_bitmap_both_ways():
    """3-D neighbour lists with and without the occupancy bitmap (it is used when
    all G^3 cell bits fit the plan's buffer: 128 bits per point of max_n)."""
    x = _blobs(77, 3000, 3, spread=14)
    for eps, max_n in ((6 / 1024, 3000), (6 / 1024, 200_000), (40 / 1024, 3000)):
        for mode in (0, 1):
            want_lab, want_cnt, want_core = oracle.dbscan(x, eps, 5, label_mode=mode)
            lab, cnt, core, st = gpu_detail(x, eps, 5, grid=B.DBSCAN_GRID_ON, label_mode=mode, max_n=max_n)
            assert st["path"] == B.DBSCAN_PATH_GRID
            np.testing.assert_array_equal(cnt, want_cnt)
            np.testing.assert_array_equal(core, want_core)
            np.testing.assert_array_equal(lab, want_lab, err_msg=f"eps={eps} max_n={max_n} mode={mode}")


# ---------------------------------------------------------------- hand-worked
def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_worked_cases(case):
    x = np.array(case["u"], dtype=np.float32) / np.float32(1024)
    eps = case["eps_units"] / 1024.0 if "eps_units" in case else case["eps_f32"]
    for g in grids_for(x.shape[1]):
        for mode, key in ((0, "labels_root"), (1, "labels_compact")):
            lab, cnt, core, _ = gpu_detail(x, eps, case["min_pts"], grid=g, label_mode=mode)
            assert lab.tolist() == case[key], (g, mode)
            assert cnt.tolist() == case["counts"]
            assert core.astype(int).tolist() == case["core"]


# ---------------------------------------------------------------- workloads
def test_small_2d_workload():
    inst = inputs.small_2d()
    assert_matches_oracle(inst.points, inst.eps, inst.min_pts)


def _blobs(seed, n, d, spread):
    rng = np.random.default_rng(seed)
    k = max(1, n // 200)
    centres = rng.integers(spread, 1024 - spread, size=(k, d))
    u = centres[rng.integers(0, k, size=n)] + rng.integers(-spread, spread + 1, size=(n, d))
    u = np.clip(u, 0, 1023)
    return (u.astype(np.float32) / np.float32(1024))


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 129, 1000, 4099])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_ragged_lowd(n, d):
    x = _blobs(100 + n + d, n, d, spread=12)
    assert_matches_oracle(x, 6 / 1024, 4)


@pytest.mark.parametrize("d", [4, 5, 7, 8, 9, 16, 17, 31, 32, 33, 64])
@pytest.mark.parametrize("n", [65, 1500])
def test_ragged_highd(n, d):
    spread = int(6 + 3 * np.sqrt(d))
    x = _blobs(200 + n + d, n, d, spread=spread)
    eps = float(np.float32(1.3 * spread * np.sqrt(d) / 1024))
    assert_matches_oracle(x, eps, 5)


@pytest.mark.parametrize("d,eps", [(17, 4.0), (32, 4.5), (64, 6.0), (8, 2.0), (16, 3.9)])
def test_huge_threshold_modes(d, eps):
    """T + 1 above 2^24 with d > 16 takes the int32 kernel; d = 8 and 16 stay in FP32."""
    rng = np.random.default_rng(d)
    u = rng.choice(np.array([0, 1, 2, 1021, 1022, 1023]), size=(300, d))
    x = u.astype(np.float32) / np.float32(1024)
    assert_matches_oracle(x, eps, 3)


def test_extreme_coordinates_near_threshold():
    """Coordinates at the grid's ends with eps put exactly on some pair distances."""
    rng = np.random.default_rng(5)
    for d in (2, 3, 8, 16):
        u = rng.choice(np.array([0, 1, 511, 512, 1022, 1023]), size=(400, d))
        x = u.astype(np.float32) / np.float32(1024)
        D = ((u[0] - u[1:]) ** 2).sum(1)
        eps = float(np.sqrt(np.median(D)) / 1024)  # float32 rounding lands T near a real D
        assert_matches_oracle(x, eps, 3)


def test_degenerate_cases():
    rng = np.random.default_rng(9)
    u = rng.integers(0, 40, size=(700, 2))
    x = u.astype(np.float32) / np.float32(1024)
    assert_matches_oracle(x, 0.5 / 1024, 2)  # T = 0: only duplicates are neighbours
    assert_matches_oracle(x, 2.0, 5)  # beyond the diameter: one cluster
    assert_matches_oracle(x, 3 / 1024, 1)  # min_pts = 1: components of the eps-graph
    assert_matches_oracle(x, 3 / 1024, 701)  # min_pts > n: all noise
    dup = np.zeros((300, 3), np.float32)  # every point identical
    assert_matches_oracle(dup, 1e-3, 5)


def test_early_exit_labels_match():
    """Without counts requested the count pass stops at min_pts; labels are unchanged."""
    inst = inputs.subsample(inputs.large_lowd(2, n=200_000), 40_000, seed=2)
    want, _, _ = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
    for g in (B.DBSCAN_GRID_ON, B.DBSCAN_GRID_OFF):
        lab, st = gpu_labels(inst.points, inst.eps, inst.min_pts, grid=g)
        np.testing.assert_array_equal(lab, want)


def test_permutation_gives_same_partition():
    inst = inputs.small_2d()
    perm = np.random.default_rng(4).permutation(inst.n)
    a, _ = gpu_labels(inst.points, inst.eps, inst.min_pts)
    b, _ = gpu_labels(inst.points[perm], inst.eps, inst.min_pts)
    back = np.empty_like(b)
    back[perm] = b
    np.testing.assert_array_equal(a == -1, back == -1)
    m = {}
    for x, y in zip(a[a >= 0], back[a >= 0]):
        assert m.setdefault(x, y) == y
    assert len(set(m.values())) == len(m)


# ---------------------------------------------------------------- API behaviour
def test_errors_and_empty():
    from paper_1506_02226_gb300.api import Plan
    with Plan(max_n=100, max_d=3) as p:
        lab = torch.empty(4, dtype=torch.int32, device="cuda")
        bad = torch.tensor([[0.25, 0.5], [0.1, 0.5], [0.5, 0.5], [0.75, 0.0]], device="cuda")
        assert B.dbscan_run(p.handle, bad.data_ptr(), 4, 2, 0.01, 2, lab.data_ptr()) == B.DBSCAN_ERR_NOT_QUANTISED
        good = torch.tensor([[0.25, 0.5]], device="cuda")
        assert B.dbscan_run(p.handle, good.data_ptr(), 0, 2, 0.01, 2, lab.data_ptr()) == B.DBSCAN_OK
        assert B.dbscan_run(p.handle, good.data_ptr(), 1, 4, 0.01, 2, lab.data_ptr()) == B.DBSCAN_ERR_ARG
        assert B.dbscan_run(p.handle, good.data_ptr(), 101, 2, 0.01, 2, lab.data_ptr()) == B.DBSCAN_ERR_ARG
        assert B.dbscan_run(p.handle, good.data_ptr(), 1, 2, 0.0, 2, lab.data_ptr()) == B.DBSCAN_ERR_ARG
        assert B.dbscan_run(p.handle, good.data_ptr(), 1, 2, float("nan"), 2, lab.data_ptr()) == B.DBSCAN_ERR_ARG
        assert B.dbscan_run(p.handle, good.data_ptr(), 1, 2, 0.01, 0, lab.data_ptr()) == B.DBSCAN_ERR_ARG
        assert B.dbscan_run(p.handle, 0, 1, 2, 0.01, 2, lab.data_ptr()) == B.DBSCAN_ERR_ARG
        # the plan is still usable after an error
        assert B.dbscan_run(p.handle, good.data_ptr(), 1, 2, 0.01, 1, lab.data_ptr()) == B.DBSCAN_OK
        assert lab[0].item() == 0
    with Plan(max_n=100, max_d=8, grid=B.DBSCAN_GRID_OFF) as p:
        bad = torch.full((10, 5), 0.3, device="cuda")
        lab = torch.empty(10, dtype=torch.int32, device="cuda")
        assert B.dbscan_run(p.handle, bad.data_ptr(), 10, 5, 0.01, 2, lab.data_ptr()) == B.DBSCAN_ERR_NOT_QUANTISED


def test_async_plan_reports_errors_on_sync():
    from paper_1506_02226_gb300.api import Plan
    inst = inputs.small_2d()
    x = torch.from_numpy(inst.points).cuda()
    want, _, _ = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
    with Plan(max_n=inst.n, max_d=2, synchronous=False) as p:
        lab = p.run(x, inst.eps, inst.min_pts)
        assert p.sync() == B.DBSCAN_OK
        np.testing.assert_array_equal(lab.cpu().numpy(), want)
        bad = x.clone()
        bad[7, 1] = 0.3
        p.run(bad, inst.eps, inst.min_pts)
        assert p.sync() == B.DBSCAN_ERR_NOT_QUANTISED
        assert p.sync() == B.DBSCAN_OK  # cleared


def test_host_entry_point_matches():
    from paper_1506_02226_gb300.api import Plan
    for inst in (inputs.small_2d(), inputs.subsample(inputs.high_d(n=20_000), 3000, seed=3)):
        want, _, _ = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
        with Plan(max_n=inst.n, max_d=inst.d) as p:
            host = torch.from_numpy(inst.points).pin_memory()
            lab = p.run_host(host, inst.eps, inst.min_pts)
        np.testing.assert_array_equal(lab.numpy(), want)


# ---------------------------------------------------------------- full size
@pytest.mark.slow
@pytest.mark.parametrize("d", [2, 3])
def test_full_size_lowd_workload(d):
    """n = 500,000 on the eps-grid path, as bench.py runs it, against the full oracle."""
    inst = inputs.large_lowd(d)
    want_lab, want_cnt, want_core = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
    lab, cnt, core, st = gpu_detail(inst.points, inst.eps, inst.min_pts)
    assert st["path"] == B.DBSCAN_PATH_GRID
    np.testing.assert_array_equal(cnt, want_cnt)
    np.testing.assert_array_equal(core, want_core)
    np.testing.assert_array_equal(lab, want_lab)
    lab2, _ = gpu_labels(inst.points, inst.eps, inst.min_pts)  # early-exit form, as timed
    np.testing.assert_array_equal(lab2, want_lab)


# ---------------------------------------------------------------- tensor-core Gram path
PRECS = [("fp16", B.DBSCAN_PREC_FP16_GRAM), ("bf16", B.DBSCAN_PREC_BF16_GRAM)]


@pytest.mark.parametrize("name,prec", PRECS)
@pytest.mark.parametrize("n,d", [(300, 16), (4099, 32), (2500, 64), (9000, 64), (1, 16), (257, 48)])
def test_tensor_core_path_matches_oracle(name, prec, n, d):
    spread = int(6 + 3 * np.sqrt(d))
    x = _blobs(300 + n + d, n, d, spread=spread)
    eps = float(np.float32(1.3 * spread * np.sqrt(d) / 1024))
    for mode in (0, 1):
        want_lab, want_cnt, want_core = oracle.dbscan(x, eps, 5, label_mode=mode)
        lab, cnt, core, st = gpu_detail(x, eps, 5, grid=B.DBSCAN_GRID_OFF, label_mode=mode, precision=prec)
        assert st["path"] == B.DBSCAN_PATH_ALLPAIRS_TC
        np.testing.assert_array_equal(cnt, want_cnt)
        np.testing.assert_array_equal(core, want_core)
        np.testing.assert_array_equal(lab, want_lab)


@pytest.mark.parametrize("name,prec", PRECS)
def test_tensor_core_dense_neighbourhoods(name, prec):
    """Almost every point core with hundreds of neighbours, several clusters that
    touch: the merge pass sees far more neighbour pairs than unions."""
    n, d = 12_000, 32
    x = _blobs(4242, n, d, spread=20)
    eps = float(np.float32(1.6 * 20 * np.sqrt(d) / 1024))
    want_lab, want_cnt, want_core = oracle.dbscan(x, eps, 8)
    assert want_core.mean() > 0.9 and np.median(want_cnt) > 50
    lab, cnt, core, st = gpu_detail(x, eps, 8, grid=B.DBSCAN_GRID_OFF, precision=prec)
    assert st["path"] == B.DBSCAN_PATH_ALLPAIRS_TC
    np.testing.assert_array_equal(cnt, want_cnt)
    np.testing.assert_array_equal(lab, want_lab)


@pytest.mark.parametrize("bf16", [0, 1])
def test_tensor_core_band_holds(bf16):
    """Every pair outside the stated rounding band is decided as exact arithmetic
    decides it; FP16 Gram products of the centred units are exact."""
    from paper_1506_02226_gb300.api import Plan
    for inst in (inputs.subsample(inputs.high_d(n=40_000), 4096, seed=5),
                 inputs.Instance(_blobs(77, 3000, 64, spread=30), 0.2, 5)):
        x = torch.from_numpy(inst.points).cuda()
        with Plan(max_n=inst.n, max_d=inst.d) as p:
            rep = B.dbscan_tc_verify(p.handle, x.data_ptr(), inst.n, inst.d, inst.eps, bf16)
        assert rep["pairs"] == inst.n ** 2
        assert rep["wrong_outside_band"] == 0
        if not bf16:
            assert rep["max_abs_error_2g"] == 0
        else:  # two-term BF16: the error bound behind the stated band (2 x 7K <= 16K)
            K = -(-inst.d // 16) * 16
            assert rep["band_halfwidth_2g"] == 16 * K
            assert rep["max_abs_error_2g"] <= 14 * K
        want = oracle.counts(inst.points, inst.eps)
        # the verify pass also counts exactly
        with Plan(max_n=inst.n, max_d=inst.d, precision=B.DBSCAN_PREC_BF16_GRAM if bf16 else
                  B.DBSCAN_PREC_FP16_GRAM, grid=B.DBSCAN_GRID_OFF) as p:
            _, cnt, _, st = p.run_detail(x, inst.eps, inst.min_pts)
        np.testing.assert_array_equal(cnt.cpu().numpy(), want)


def test_tensor_core_high_d_subsample():
    inst = inputs.subsample(inputs.high_d(n=60_000), 12_000, seed=8)
    want_lab, want_cnt, want_core = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
    for prec in (B.DBSCAN_PREC_FP16_GRAM, B.DBSCAN_PREC_BF16_GRAM, B.DBSCAN_PREC_EXACT_SIMT):
        lab, cnt, core, st = gpu_detail(inst.points, inst.eps, inst.min_pts, grid=B.DBSCAN_GRID_OFF,
                                        precision=prec)
        np.testing.assert_array_equal(cnt, want_cnt)
        np.testing.assert_array_equal(lab, want_lab)


@pytest.mark.slow
def test_full_size_high_d_workload():
    """n = 200,000, d = 64 on the FP16 and the two-term BF16 tensor-core paths,
    against the full oracle."""
    from paper_1506_02226_gb300.api import Plan
    inst = inputs.high_d()
    want_lab, want_cnt, want_core = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
    lab, cnt, core, st = gpu_detail(inst.points, inst.eps, inst.min_pts)
    assert st["path"] == B.DBSCAN_PATH_ALLPAIRS_TC
    np.testing.assert_array_equal(cnt, want_cnt)
    np.testing.assert_array_equal(core, want_core)
    np.testing.assert_array_equal(lab, want_lab)
    lab2, _ = gpu_labels(inst.points, inst.eps, inst.min_pts)
    np.testing.assert_array_equal(lab2, want_lab)
    lab3, cnt3, core3, st3 = gpu_detail(inst.points, inst.eps, inst.min_pts, precision=B.DBSCAN_PREC_BF16_GRAM)
    assert st3["path"] == B.DBSCAN_PATH_ALLPAIRS_TC and st3["band_pairs"] > 0
    np.testing.assert_array_equal(cnt3, want_cnt)
    np.testing.assert_array_equal(lab3, want_lab)
    x = torch.from_numpy(inst.points).cuda()
    with Plan(max_n=inst.n, max_d=inst.d, precision=B.DBSCAN_PREC_BF16_GRAM) as p:  # as bench.py times it
        np.testing.assert_array_equal(p.run(x, inst.eps, inst.min_pts).cpu().numpy(), want_lab)


def test_tensor_core_plan_reused_across_sizes():
    """One plan, instances of shrinking size: nothing of an earlier run may leak
    into a later one (counters, packed operands, set hints)."""
    from paper_1506_02226_gb300.api import Plan
    with Plan(max_n=12_000, max_d=32, precision=B.DBSCAN_PREC_FP16_GRAM, grid=B.DBSCAN_GRID_OFF) as p:
        for seed, n, d in ((1, 11_000, 16), (2, 7519, 16), (3, 3000, 32), (4, 500, 16), (5, 9000, 32)):
            spread = int(6 + 3 * np.sqrt(d))
            x = _blobs(seed, n, d, spread=spread)
            eps = float(np.float32(1.3 * spread * np.sqrt(d) / 1024))
            lab, cnt, core, st = p.run_detail(torch.from_numpy(x).cuda(), eps, 6)
            want_lab, want_cnt, _ = oracle.dbscan(x, eps, 6)
            np.testing.assert_array_equal(cnt.cpu().numpy(), want_cnt)
            np.testing.assert_array_equal(lab.cpu().numpy(), want_lab)


def test_grid_run_captured_in_a_cuda_graph():
    """An asynchronous plan's run (the eps-grid path, whose independent kernels
    fork onto the plan's second stream and join back) captured into a CUDA graph
    and replayed on new data of the same shape."""
    from paper_1506_02226_gb300.api import Plan
    a = _blobs(501, 20_000, 2, spread=12)
    b = _blobs(502, 20_000, 2, spread=12)
    eps, mp = 6 / 1024, 5
    s = torch.cuda.Stream()
    x = torch.from_numpy(a).cuda()
    lab = torch.empty(a.shape[0], dtype=torch.int32, device="cuda")
    with Plan(max_n=a.shape[0], max_d=2, synchronous=False, stream=s) as p:
        with torch.cuda.stream(s):
            p.run(x, eps, mp, labels=lab)  # warm-up outside the capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            p.run(x, eps, mp, labels=lab)
        for pts in (a, b):
            x.copy_(torch.from_numpy(pts))
            g.replay()
            torch.cuda.synchronize()
            assert p.sync() == B.DBSCAN_OK
            np.testing.assert_array_equal(lab.cpu().numpy(), oracle.dbscan(pts, eps, mp)[0])
