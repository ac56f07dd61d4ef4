"""Served form: continuous batching, results identical alone and in the mix."""
import threading

import numpy as np
import pytest

import oracle
from paper_1506_02226_gb300 import binding as B
from paper_1506_02226_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _jobs(count, n_max, seed=0):
    out = []
    for i in range(count):
        inst = inputs.serve_job(i, seed=inputs.SEED_BASE + 5 + seed, n_max=n_max)
        x = torch.from_numpy(inst.points).cuda()
        lab = torch.full((inst.n,), -9, dtype=torch.int32, device="cuda")
        out.append((inst, x, lab))
    return out


def _instance(inst, x, lab):
    s = B.dbscan_instance()
    s.points = x.data_ptr()
    s.n = inst.n
    s.d = inst.d
    s.eps = inst.eps
    s.min_pts = inst.min_pts
    s.labels_out = lab.data_ptr()
    return s


def _alone(jobs):
    from paper_1506_02226_gb300.api import Plan
    out = []
    with Plan(max_n=max(j[0].n for j in jobs), max_d=64) as p:
        for inst, x, _ in jobs:
            out.append(p.run(x, inst.eps, inst.min_pts).cpu().numpy())
    return out


def _serve(jobs, slots=4, budget=None, threads=2):
    o = B.dbscan_serve_opts_default()
    o.slots = slots
    o.max_n = max(j[0].n for j in jobs)
    if budget is not None:
        o.hbm_budget_bytes = budget
    srv = B.dbscan_serve_create(o)
    ids = [None] * len(jobs)
    structs = [_instance(*j) for j in jobs]

    def submit(part):
        for k in part:
            ids[k] = B.dbscan_serve_submit(srv, structs[k])

    ts = [threading.Thread(target=submit, args=(range(t, len(jobs), threads),)) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    res = []
    for k in range(len(jobs)):
        st, lat = B.dbscan_serve_wait(srv, ids[k], -1)
        res.append((st, lat))
    B.dbscan_serve_destroy(srv)
    return res


def test_serve_results_identical_alone_and_in_mix():
    jobs = _jobs(48, n_max=30_000)
    want = _alone(jobs)
    res = _serve(jobs, slots=6, threads=3)
    for k, ((inst, x, lab), (st, lat)) in enumerate(zip(jobs, res)):
        assert st == B.DBSCAN_OK
        assert lat > 0
        np.testing.assert_array_equal(lab.cpu().numpy(), want[k], err_msg=f"job {k} n={inst.n} d={inst.d}")
    for (inst, x, lab) in jobs[:6]:
        np.testing.assert_array_equal(lab.cpu().numpy(), oracle.dbscan(inst.points, inst.eps, inst.min_pts)[0])


def test_serve_tight_budget_still_completes():
    jobs = _jobs(12, n_max=20_000, seed=1)
    want = _alone(jobs)
    res = _serve(jobs, slots=4, budget=1, threads=1)  # one job on the device at a time
    for (inst, x, lab), w, (st, _) in zip(jobs, want, res):
        assert st == B.DBSCAN_OK
        np.testing.assert_array_equal(lab.cpu().numpy(), w)


def test_serve_errors():
    o = B.dbscan_serve_opts_default()
    o.slots = 2
    o.max_n = 1000
    srv = B.dbscan_serve_create(o)
    try:
        good = _jobs(1, n_max=1000)[0]
        bad_pts = torch.full((50, 2), 0.3, device="cuda")
        bad_lab = torch.empty(50, dtype=torch.int32, device="cuda")
        bad = B.dbscan_instance()
        bad.points, bad.n, bad.d, bad.eps, bad.min_pts, bad.labels_out = (bad_pts.data_ptr(), 50, 2, 0.01, 3,
                                                                          bad_lab.data_ptr())
        jb = B.dbscan_serve_submit(srv, bad)
        jg = B.dbscan_serve_submit(srv, _instance(*good))
        assert B.dbscan_serve_wait(srv, jb, -1)[0] == B.DBSCAN_ERR_NOT_QUANTISED
        assert B.dbscan_serve_wait(srv, jg, -1)[0] == B.DBSCAN_OK  # a bad job does not spoil the others
        np.testing.assert_array_equal(good[2].cpu().numpy(), _alone([good])[0])
        big = B.dbscan_instance()
        big.points, big.n, big.d, big.eps, big.min_pts, big.labels_out = bad.points, 5000, 2, 0.01, 3, bad.labels_out
        with pytest.raises(B.DbscanError):
            B.dbscan_serve_submit(srv, big)  # n > max_n
        assert B.dbscan_serve_wait(srv, 987654321, 0)[0] == B.DBSCAN_ERR_NOT_FOUND
        assert B.dbscan_serve_poll(srv, 987654321)[0] == B.DBSCAN_ERR_NOT_FOUND
    finally:
        B.dbscan_serve_destroy(srv)


@pytest.mark.slow
def test_serve_bench_job_pool_alone_and_in_mix():
    """The 192 seeded jobs bench.py's served workload cycles (n up to 500k, d in
    {2, 3, 32}): each result in the mix equals the same job run alone, and the
    smaller jobs equal the oracle."""
    jobs = []
    for i in range(192):
        inst = inputs.serve_job(i)
        x = torch.from_numpy(inst.points).cuda()
        jobs.append((inst, x, torch.full((inst.n,), -9, dtype=torch.int32, device="cuda")))
    want = _alone(jobs)
    res = _serve(jobs, slots=8, threads=4)
    for k, ((inst, x, lab), (st, _)) in enumerate(zip(jobs, res)):
        assert st == B.DBSCAN_OK
        np.testing.assert_array_equal(lab.cpu().numpy(), want[k], err_msg=f"job {k} n={inst.n} d={inst.d}")
    # every job up to 20,000 points and ten larger ones (seeded pick up to 120,000) against the oracle
    small = [j for j in jobs if j[0].n <= 20_000]
    larger = [j for j in jobs if 20_000 < j[0].n <= 120_000]
    pick = np.random.default_rng(7).choice(len(larger), size=min(10, len(larger)), replace=False)
    assert len(small) >= 100 and len(pick) == 10
    for inst, x, lab in small + [larger[i] for i in pick]:
        np.testing.assert_array_equal(lab.cpu().numpy(), oracle.dbscan(inst.points, inst.eps, inst.min_pts)[0],
                                      err_msg=f"n={inst.n} d={inst.d}")


def _copies(inst, count):
    x = torch.from_numpy(inst.points).cuda()
    return [(inst, x, torch.full((inst.n,), -9, dtype=torch.int32, device="cuda")) for _ in range(count)]


def _serve_stats(jobs, slots, budget):
    o = B.dbscan_serve_opts_default()
    o.slots = slots
    o.max_n = max(j[0].n for j in jobs)
    o.hbm_budget_bytes = budget
    srv = B.dbscan_serve_create(o)
    try:
        structs = [_instance(*j) for j in jobs]
        ids = [B.dbscan_serve_submit(srv, s) for s in structs]
        sts = [B.dbscan_serve_wait(srv, i, -1)[0] for i in ids]
        info = B.dbscan_serve_info(srv)
        per_job = B.dbscan_serve_job_bytes(srv, jobs[0][0].n, jobs[0][0].d)
    finally:
        B.dbscan_serve_destroy(srv)
    return sts, info, per_job


def test_serve_budget_limits_concurrency_by_bytes():
    """Eight equal jobs on eight slots: the budget, not the slot count, decides
    how many run at once, and the bytes on the device stay within it."""
    base = inputs.serve_job(3, seed=inputs.SEED_BASE + 77, n_max=60_000)
    inst = inputs.Instance(np.ascontiguousarray(base.points), base.eps, base.min_pts)
    want = _alone([(inst, torch.from_numpy(inst.points).cuda(), None)])[0]
    o = B.dbscan_serve_opts_default()
    o.max_n = inst.n + 10
    probe = B.dbscan_serve_create(o)
    job = B.dbscan_serve_job_bytes(probe, inst.n, inst.d)
    assert B.dbscan_serve_job_bytes(probe, inst.n + 1, inst.d) >= job > 0
    assert B.dbscan_serve_job_bytes(probe, o.max_n + 1, inst.d) == -1
    B.dbscan_serve_destroy(probe)
    for k, expect_max in ((1, 1), (3, 3), (1000, 8)):
        jobs = _copies(inst, 8)
        budget = int(job * (k + 0.5))
        sts, info, per_job = _serve_stats(jobs, slots=8, budget=budget)
        assert per_job == job
        assert all(st == B.DBSCAN_OK for st in sts)
        assert info["jobs_done"] == 8 and info["jobs_running"] == 0 and info["bytes_in_flight"] == 0
        assert 1 <= info["max_jobs_running"] <= expect_max, (k, info)
        assert info["peak_bytes_in_flight"] <= budget and info["peak_bytes_in_flight"] == info["max_jobs_running"] * job
        if k < 8:  # the pool holds about what the admitted jobs use, not the slot count's worth
            assert info["pool_peak_reserved_bytes"] <= budget + (64 << 20), (k, info)
        else:
            assert info["max_jobs_running"] >= 2, info
        for inst_, x, lab in jobs:
            np.testing.assert_array_equal(lab.cpu().numpy(), want)


def test_serve_destroy_while_another_thread_waits():
    """dbscan_serve_destroy while a thread is blocked in dbscan_serve_wait: the
    waiter returns (its job ran or was dropped) before anything is freed."""
    jobs = _jobs(10, n_max=40_000, seed=3)
    o = B.dbscan_serve_opts_default()
    o.slots = 2
    o.max_n = max(j[0].n for j in jobs)
    srv = B.dbscan_serve_create(o)
    ids = [B.dbscan_serve_submit(srv, _instance(*j)) for j in jobs]
    got = {}

    def waiter():
        got["st"] = B.dbscan_serve_wait(srv, ids[-1], -1)[0]

    t = threading.Thread(target=waiter)
    t.start()
    B.dbscan_serve_destroy(srv)
    t.join(timeout=60)
    assert not t.is_alive()
    assert got["st"] in (B.DBSCAN_OK, B.DBSCAN_ERR_BUSY)
