"""Batched form (dbscan_batch) against the oracle, instance by instance, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1506_02226_gb300 import binding as B
from paper_1506_02226_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mixed_instances(seed, count, dims=(1, 2, 3, 5, 8, 16), nmax=3000):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(0, nmax)) if i % 7 else int(rng.integers(0, 3))  # some empty / tiny
        d = int(rng.choice(dims))
        k = int(rng.integers(1, 6))
        spread = int(rng.integers(5, 40))
        centres = rng.integers(spread, 1024 - spread, size=(k, d))
        u = centres[rng.integers(0, k, size=n)] + rng.integers(-spread, spread + 1, size=(n, d))
        x = (np.clip(u, 0, 1023).astype(np.float32) / np.float32(1024)).reshape(n, d)
        eps = float(np.float32(rng.uniform(0.5, 1.5) * spread * np.sqrt(d) / 1024))
        out.append(inputs.Instance(x, eps, int(rng.integers(1, 12))))
    return out


def _run_batch(plan, insts, stats=False):
    from paper_1506_02226_gb300.api import make_instances
    items = []
    for inst in insts:
        x = torch.from_numpy(np.ascontiguousarray(inst.points)).cuda() if inst.n else \
            torch.zeros((1, inst.d), device="cuda")
        lab = torch.full((max(inst.n, 1),), -9, dtype=torch.int32, device="cuda")
        items.append((x, inst.eps, inst.min_pts, lab))
    arr = make_instances(items)
    for k, inst in enumerate(insts):
        arr[k].n = inst.n
        arr[k].d = inst.d
    st = (B.dbscan_stats * len(insts))() if stats else None
    rc = B.dbscan_batch(plan.handle, arr, st)
    return rc, [it[3][:inst.n].cpu().numpy() for it, inst in zip(items, insts)], st


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_matches_oracle(mode):
    from paper_1506_02226_gb300.api import Plan
    insts = _mixed_instances(11 + mode, 60)
    with Plan(max_n=16, max_d=16, label_mode=mode) as p:
        rc, labs, st = _run_batch(p, insts, stats=True)
        assert rc == B.DBSCAN_OK
        for k, (inst, lab) in enumerate(zip(insts, labs)):
            want, _, core = oracle.dbscan(inst.points, inst.eps, inst.min_pts, label_mode=mode)
            np.testing.assert_array_equal(lab, want, err_msg=f"instance {k} n={inst.n} d={inst.d}")
            assert st[k].n_core == int(core.sum())
            assert st[k].n_core + st[k].n_border + st[k].n_noise == inst.n
            assert st[k].n_clusters == len(set(want[want >= 0].tolist()))
        ch, bps = B.dbscan_batch_config(p.handle)
        assert ch > 0 and bps > 0
        assert B.dbscan_batch_tile(p.handle) in ((32, 64), (64, 64), (128, 64))


def test_batch_graph_reuse_and_growth():
    """Second call reuses the captured graph on new data; a larger batch grows the workspace."""
    from paper_1506_02226_gb300.api import Plan
    with Plan(max_n=16, max_d=16) as p:
        for seed, count in ((21, 40), (22, 40), (23, 150)):
            insts = _mixed_instances(seed, count, nmax=2500)
            rc, labs, _ = _run_batch(p, insts)
            assert rc == B.DBSCAN_OK
            for inst, lab in zip(insts, labs):
                want, _, _ = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
                np.testing.assert_array_equal(lab, want)


def test_batch_workload_sample_matches_dbscan_run():
    """A slice of the 4,096-instance workload: batch labels equal per-instance dbscan_run labels."""
    from paper_1506_02226_gb300.api import Plan
    insts = inputs.batch(count=256)
    with Plan(max_n=8192, max_d=16) as single, Plan(max_n=16, max_d=16) as bp:
        rc, labs, _ = _run_batch(bp, insts)
        assert rc == B.DBSCAN_OK
        for k, (inst, lab) in enumerate(zip(insts, labs)):
            x = torch.from_numpy(inst.points).cuda()
            want = single.run(x, inst.eps, inst.min_pts).cpu().numpy()
            np.testing.assert_array_equal(lab, want, err_msg=f"instance {k}")
        for inst, lab in list(zip(insts, labs))[:24]:
            np.testing.assert_array_equal(lab, oracle.dbscan(inst.points, inst.eps, inst.min_pts)[0])


def test_batch_errors():
    from paper_1506_02226_gb300.api import Plan
    with Plan(max_n=16, max_d=16) as p:
        good = _mixed_instances(5, 3)
        bad = inputs.Instance(np.full((10, 2), 0.3, np.float32), 0.01, 3)
        rc, _, _ = _run_batch(p, good + [bad])
        assert rc == B.DBSCAN_ERR_NOT_QUANTISED
        wide = inputs.Instance(np.zeros((10, 17), np.float32), 0.01, 3)
        rc, _, _ = _run_batch(p, [wide])
        assert rc == B.DBSCAN_ERR_UNSUPPORTED
        rc, labs, _ = _run_batch(p, good)  # usable after errors
        assert rc == B.DBSCAN_OK
        for inst, lab in zip(good, labs):
            np.testing.assert_array_equal(lab, oracle.dbscan(inst.points, inst.eps, inst.min_pts)[0])


@pytest.mark.slow
def test_full_batch_workload_against_oracle():
    """All 4,096 instances in one dbscan_batch call, as bench.py runs it; every
    7th instance against dbscan_run alone and every instance against the oracle."""
    from paper_1506_02226_gb300.api import Plan
    insts = inputs.batch(count=4096)
    with Plan(max_n=16, max_d=16) as bp:
        rc, labs, st = _run_batch(bp, insts, stats=True)
        assert rc == B.DBSCAN_OK
    with Plan(max_n=8192, max_d=16) as single:
        for k in range(0, 4096, 7):  # every 7th instance against a plain run
            inst = insts[k]
            want = single.run(torch.from_numpy(inst.points).cuda(), inst.eps, inst.min_pts).cpu().numpy()
            np.testing.assert_array_equal(labs[k], want, err_msg=f"instance {k}")
    for k, inst in enumerate(insts):
        want, _, core = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
        np.testing.assert_array_equal(labs[k], want, err_msg=f"instance {k}")
        assert st[k].n_core == int(core.sum())
        assert st[k].n_core + st[k].n_border + st[k].n_noise == inst.n
        assert 0 < st[k].pair_tests <= 3 * inst.n * inst.n + 64 * 64
