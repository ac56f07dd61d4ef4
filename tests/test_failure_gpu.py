"""Failure detection without a GPU fault: bounded device waits that expire on
purpose (a test hook stalls the tensor-core MMA issue), an allocation that
cannot succeed, and the plan staying usable after each."""
import numpy as np
import pytest

import oracle
from paper_1506_02226_gb300 import binding as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _blobs(seed, n, d, spread):
    rng = np.random.default_rng(seed)
    centres = rng.integers(spread, 1024 - spread, size=(max(1, n // 300), d))
    u = centres[rng.integers(0, len(centres), size=n)] + rng.integers(-spread, spread + 1, size=(n, d))
    return np.clip(u, 0, 1023).astype(np.float32) / np.float32(1024)


def test_tensor_core_wait_expiry_reports_timeout_and_plan_recovers():
    from paper_1506_02226_gb300.api import Plan
    n, d = 5000, 32
    x = _blobs(7, n, d, spread=20)
    eps = float(np.float32(1.3 * 20 * np.sqrt(d) / 1024))
    xd = torch.from_numpy(x).cuda()
    with Plan(max_n=n, max_d=d, precision=B.DBSCAN_PREC_FP16_GRAM, grid=B.DBSCAN_GRID_OFF) as p:
        B.dbscan_plan_test_hook(p.handle, B.DBSCAN_HOOK_TC_STALL)
        with pytest.raises(B.DbscanError) as err:
            p.run(xd, eps, 6)
        assert err.value.status == B.DBSCAN_ERR_TIMEOUT
        # the hook was consumed: the same plan clusters correctly again
        lab = p.run(xd, eps, 6).cpu().numpy()
        np.testing.assert_array_equal(lab, oracle.dbscan(x, eps, 6)[0])


def test_test_hook_rejects_unknown_values():
    from paper_1506_02226_gb300.api import Plan
    with Plan(max_n=16, max_d=2) as p:
        with pytest.raises(B.DbscanError) as err:
            B.dbscan_plan_test_hook(p.handle, 99)
        assert err.value.status == B.DBSCAN_ERR_ARG
        B.dbscan_plan_test_hook(p.handle, B.DBSCAN_HOOK_NONE)


def test_allocation_failure_reports_oom_and_leaves_the_device_usable():
    from paper_1506_02226_gb300.api import Plan
    with pytest.raises(B.DbscanError) as err:
        Plan(max_n=(2**31 - 1) // 2, max_d=64)  # a workspace far beyond the device's memory
    assert err.value.status == B.DBSCAN_ERR_OOM
    x = _blobs(3, 1000, 2, spread=10)
    with Plan(max_n=1000, max_d=2) as p:
        lab = p.run(torch.from_numpy(x).cuda(), 5 / 1024, 4).cpu().numpy()
    np.testing.assert_array_equal(lab, oracle.dbscan(x, 5 / 1024, 4)[0])
