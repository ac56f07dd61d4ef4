"""The paper's own materialised pipeline (comparison variant) against the oracle.

dbscan_run_paper builds the N x N distance matrix, the primitive-cluster
matrix and the `valid` vector, and merges clusters by one launch per target
(Section IV), sweeping until nothing merges; its labels must equal the
oracle's (and so dbscan_run's) bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1506_02226_gb300 import binding as B
from paper_1506_02226_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def paper_labels(points, eps, min_pts, label_mode=0):
    from paper_1506_02226_gb300.api import Plan
    n, d = points.shape
    x = torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).cuda()
    with Plan(max_n=max(n, 1), max_d=max(d, 1), label_mode=label_mode) as p:
        lab, st = p.run_paper(x, eps, min_pts, stats=True)
    return lab.cpu().numpy(), st


def check(points, eps, min_pts):
    for mode in (0, 1):
        want, _, core = oracle.dbscan(points, eps, min_pts, label_mode=mode)
        got, st = paper_labels(points, eps, min_pts, label_mode=mode)
        np.testing.assert_array_equal(got, want, err_msg=f"mode={mode}")
        assert st["path"] == B.DBSCAN_PATH_PAPER
        assert st["n_core"] == int(core.sum()) and st["n_core"] + st["n_border"] + st["n_noise"] == len(want)
        assert st["cells"] >= 1  # merge sweeps
        assert st["pair_tests"] == len(want) ** 2


def blobs(seed, n, d, spread):
    rng = np.random.default_rng(seed)
    centres = rng.integers(60, 960, size=(6, d))
    u = np.clip(centres[rng.integers(0, 6, size=n)] + rng.integers(-spread, spread + 1, size=(n, d)), 0, 1023)
    noise = rng.random(n) < 0.1
    u[noise] = rng.integers(0, 1024, size=(int(noise.sum()), d))
    return u.astype(np.float32) / np.float32(1024)


def test_small_2d_workload():
    inst = inputs.small_2d()
    check(inst.points, inst.eps, inst.min_pts)


@pytest.mark.parametrize("n,d", [(1, 2), (2, 3), (127, 3), (129, 3), (3000, 3), (1500, 8), (900, 16)])
def test_blobs(n, d):
    x = blobs(n + d, n, d, spread=int(10 + 3 * np.sqrt(d)))
    check(x, float(np.float32(1.2 * (10 + 3 * np.sqrt(d)) * np.sqrt(d) / 1024)), 4)


def test_chains_need_several_merges():
    """A long chain of cores in index order reversed: merges reach the first
    target only through later ones, so the sweep repeats."""
    n = 400
    u = np.zeros((n, 2), np.int64)
    u[:, 0] = np.arange(n)[::-1] * 2  # neighbours two units apart along x, indices descending
    x = u.astype(np.float32) / np.float32(1024)
    check(x, 2.5 / 1024, 2)


def test_degenerate_cases():
    rng = np.random.default_rng(3)
    x = (rng.integers(0, 40, size=(600, 3)).astype(np.float32) / np.float32(1024))
    check(x, 0.5 / 1024, 2)  # T = 0
    check(x, 2.0, 5)  # one cluster
    check(x, 3 / 1024, 1)  # components
    check(x, 3 / 1024, 601)  # all noise
    check(np.zeros((300, 2), np.float32), 1e-3, 5)


def test_errors():
    from paper_1506_02226_gb300.api import Plan
    with Plan(max_n=100, max_d=32) as p:
        x = torch.zeros((10, 20), device="cuda")
        lab = torch.empty(10, dtype=torch.int32, device="cuda")
        assert B.dbscan_run_paper(p.handle, x.data_ptr(), 10, 20, 0.01, 2, lab.data_ptr()) == B.DBSCAN_ERR_ARG
        bad = torch.full((10, 2), 0.3, device="cuda")
        assert B.dbscan_run_paper(p.handle, bad.data_ptr(), 10, 2, 0.01, 2, lab.data_ptr()) == \
            B.DBSCAN_ERR_NOT_QUANTISED
        assert B.dbscan_run_paper(p.handle, x.data_ptr(), 0, 2, 0.01, 2, lab.data_ptr()) == B.DBSCAN_OK
