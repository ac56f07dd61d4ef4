"""dbscan_run_noalloc, the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc, for example a service that reserved all
device memory for its own pool, or code that must not take the allocator's
locks.  dbscan_run_noalloc takes its scratch from a fixed array inside the
library instead of a plan.  These tests call it through the C ABI twice in a
row and check each result against dbscan_run's on the same input and against
the oracle; labels are integers from an exact predicate, so they must be equal.
The calls run largest first (one at the array's size limit), so each later
call runs over scratch a larger call left behind.  This file is collected
last, so that a run stopping at the first failure has run every other test
first.
"""
import numpy as np
import pytest

import oracle
from paper_1506_02226_gb300 import binding as B
from paper_1506_02226_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _with_plan(x, eps, min_pts, label_mode):
    from paper_1506_02226_gb300.api import Plan
    with Plan(max_n=x.shape[0], max_d=x.shape[1], label_mode=label_mode) as p:
        return p.run(x, eps, min_pts).cpu().numpy()


def _noalloc(x, eps, min_pts, label_mode):
    n, d = x.shape
    lab = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    rc = B.dbscan_run_noalloc(x.data_ptr(), n, d, eps, min_pts, label_mode, lab.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert rc == B.DBSCAN_OK, B.dbscan_strerror(rc)
    return lab.cpu().numpy()


def _random_instance(seed, n, d):
    rng = np.random.default_rng(seed)
    centres = rng.integers(100, 900, size=(6, d))
    u = np.clip(centres[rng.integers(0, 6, size=n)] + rng.integers(-40, 41, size=(n, d)), 0, 1023)
    return u.astype(np.float32) / np.float32(1024)


def test_noalloc_matches_dbscan_run_two_calls_in_a_row():
    small = inputs.small_2d()
    cases = [  # largest first: later calls run over what a larger call left in the shared scratch
        (_random_instance(7, B.DBSCAN_NOALLOC_MAX_N, B.DBSCAN_NOALLOC_MAX_D), 0.08, 8, B.DBSCAN_LABEL_ROOT_INDEX),
        (_random_instance(3, 9000, 16), 0.09, 6, B.DBSCAN_LABEL_COMPACT),
        (small.points, small.eps, small.min_pts, B.DBSCAN_LABEL_ROOT_INDEX),
        (small.points, small.eps, small.min_pts, B.DBSCAN_LABEL_COMPACT),
    ]
    for pts, eps, mp, mode in cases:  # back to back: the shared scratch holds the previous call's data
        x = torch.from_numpy(pts).cuda()
        got = _noalloc(x, eps, mp, mode)
        want = _with_plan(x, eps, mp, mode)
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(got, oracle.dbscan(pts, eps, mp, label_mode=mode)[0])
        assert (got >= 0).any() and (got == -1).any()


def test_noalloc_limits_and_errors():
    x = torch.zeros((B.DBSCAN_NOALLOC_MAX_N + 1, 2), device="cuda")
    lab = torch.empty(x.shape[0], dtype=torch.int32, device="cuda")
    assert B.dbscan_run_noalloc(x.data_ptr(), x.shape[0], 2, 0.01, 3, 0, lab.data_ptr(), None) == B.DBSCAN_ERR_ARG
    assert B.dbscan_run_noalloc(x.data_ptr(), 10, B.DBSCAN_NOALLOC_MAX_D + 1, 0.01, 3, 0, lab.data_ptr(),
                                None) == B.DBSCAN_ERR_ARG
    bad = torch.full((10, 2), 0.3, device="cuda")
    assert B.dbscan_run_noalloc(bad.data_ptr(), 10, 2, 0.01, 3, 0, lab.data_ptr(), None) == \
        B.DBSCAN_ERR_NOT_QUANTISED
    assert B.dbscan_run_noalloc(x.data_ptr(), 0, 2, 0.01, 3, 0, lab.data_ptr(), None) == B.DBSCAN_OK
