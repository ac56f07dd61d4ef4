"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test ties the oracle to the paper's definitions (Section II), to a
textbook or library routine for a special case, to an independent
implementation, or to hand-worked values in tests/golden/hand_cases.json.
The planted-mistake test shows that the pins fail when the oracle is wrong in
a plausible way.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.bfs import dbscan_bfs, neighbour_lists
from paper_1506_02226_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def _case_input(c):
    x = np.array(c["u"], dtype=np.float32) / np.float32(1024)
    eps = c["eps_units"] / 1024.0 if "eps_units" in c else c["eps_f32"]
    return x, float(np.float32(eps))


def _check_case(c, mutation=0):
    x, eps = _case_input(c)
    ok = True
    for mode, key in ((0, "labels_root"), (1, "labels_compact")):
        lab, cnt, core = oracle.dbscan(x, eps, c["min_pts"], label_mode=mode, mutation=mutation)
        ok &= lab.tolist() == c[key]
        ok &= cnt.tolist() == c["counts"]
        ok &= core.astype(int).tolist() == c["core"]
    return ok


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_worked_cases(case):
    assert _check_case(case)
    if "T" in case:
        assert oracle.threshold(_case_input(case)[1]) == case["T"]


def test_planted_mistakes_are_caught():
    """Each planted mistake in the oracle fails at least one hand-worked case."""
    for mut in (oracle.MUT_STRICT_LESS, oracle.MUT_NO_SELF, oracle.MUT_BORDER_MAX, oracle.MUT_NO_UNION):
        assert not all(_check_case(c, mutation=mut) for c in _cases()), mut


@pytest.mark.parametrize("eps", [0.02, 0.005, 0.4566502869129181, 1e-4, 3 / 1024, 0.123456789, 1.5])
def test_threshold_is_exact_floor(eps):
    """T = floor(eps^2 * 2^20) for the float32 eps, checked in exact rationals."""
    e = Fraction(float(np.float32(eps)))
    assert oracle.threshold(eps) == math.floor(e * e * 2 ** 20)


@pytest.mark.parametrize("bad", [1e-4, -1 / 1024, 1.0, 2.0, float("nan"), float("inf"), 0.5 + 2 ** -11])
def test_quantisation_rejects_off_grid(bad):
    x = np.array([[0.25, 0.5], [bad, 0.125]], dtype=np.float32)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.dbscan(x, 0.01, 2)
    assert ei.value.status == oracle.ERR_NOT_QUANTISED


def _random_grid(rng, n, d, spread=1024, lo=0):
    u = rng.integers(lo, lo + spread, size=(n, d))
    return (u.astype(np.float32) / np.float32(1024)), u


def _canon_components(n, pairs):
    """Connected components (scipy) relabelled by their smallest member."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    if len(pairs):
        p = np.array(sorted(pairs))
        g = coo_matrix((np.ones(len(p)), (p[:, 0], p[:, 1])), shape=(n, n))
    else:
        g = coo_matrix((n, n))
    _, comp = connected_components(g, directed=False)
    first = {}
    for i, c in enumerate(comp):
        first.setdefault(c, i)
    return np.array([first[c] for c in comp])


@pytest.mark.parametrize("seed,n,d,eps_u", [(1, 300, 2, 20), (2, 400, 3, 60), (3, 250, 1, 3),
                                            (4, 200, 5, 150), (5, 300, 2, 7)])
def test_min_pts_one_is_connected_components(seed, n, d, eps_u):
    """min_pts = 1 makes every point core: labels = components of the eps-graph.

    The eps-graph comes from scipy's k-d tree on the integer units with radius
    sqrt(T + 1/2), which separates D <= T from D >= T + 1 for integer D.
    """
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    x, u = _random_grid(rng, n, d, spread=200)
    eps = eps_u / 1024.0
    T = oracle.threshold(eps)
    pairs = cKDTree(u.astype(np.float64)).query_pairs(math.sqrt(T + 0.5))
    want = _canon_components(n, pairs)
    lab, _, core = oracle.dbscan(x, eps, 1)
    assert core.all()
    np.testing.assert_array_equal(lab, want)


def test_eps_above_diameter_gives_one_cluster():
    rng = np.random.default_rng(7)
    for d in (1, 2, 3, 8):
        x, _ = _random_grid(rng, 150, d)
        eps = float(np.float32(math.sqrt(d) + 0.01))  # beyond the diagonal of [0,1)^d
        lab, cnt, core = oracle.dbscan(x, eps, 10)
        assert (cnt == 150).all() and core.all() and (lab == 0).all()
        lab, _, _ = oracle.dbscan(x, eps, 10, label_mode=1)
        assert (lab == 0).all()


def test_min_pts_above_n_is_all_noise():
    rng = np.random.default_rng(8)
    x, _ = _random_grid(rng, 120, 2, spread=50)
    lab, _, core = oracle.dbscan(x, 0.05, 121)
    assert (lab == -1).all() and not core.any()


def test_empty_input():
    lab, cnt, core = oracle.dbscan(np.zeros((0, 3), np.float32), 0.1, 3)
    assert lab.shape == (0,)


def _check_against_bfs(x, eps, min_pts):
    classic, canon, core_b = dbscan_bfs(x, eps, min_pts)
    lab, cnt, core = oracle.dbscan(x, eps, min_pts)
    np.testing.assert_array_equal(core, core_b)
    np.testing.assert_array_equal(lab, canon)
    # The classic first-come border assignment is a valid DBSCAN result too:
    # same core partition, and each border point sits in a cluster of one of
    # its core neighbours.
    np.testing.assert_array_equal(lab[core], classic[core])
    nb = neighbour_lists(x, eps)
    for p in np.nonzero(~core)[0]:
        cn = [q for q in nb[p] if core[q]]
        if cn:
            assert classic[p] in {lab[q] for q in cn}
        else:
            assert classic[p] == -1 and lab[p] == -1


def test_against_independent_bfs_small_2d_workload():
    inst = inputs.small_2d()
    _check_against_bfs(inst.points, inst.eps, inst.min_pts)


@pytest.mark.parametrize("seed,n,d,spread,eps_u,min_pts", [
    (11, 500, 2, 128, 6, 4),  # dense: many border ties
    (12, 400, 3, 64, 5, 6),
    (13, 300, 1, 200, 2, 3),  # 1-D chains at exactly eps
    (14, 300, 2, 16, 1, 5),  # lots of duplicates
    (15, 200, 16, 64, 60, 3),
])
def test_against_independent_bfs_random(seed, n, d, spread, eps_u, min_pts):
    rng = np.random.default_rng(seed)
    x, _ = _random_grid(rng, n, d, spread=spread)
    _check_against_bfs(x, eps_u / 1024.0, min_pts)


def test_against_sklearn():
    """Core sets, the partition of core points and the noise set match sklearn."""
    skc = pytest.importorskip("sklearn.cluster")
    cases = [inputs.small_2d(), inputs.subsample(inputs.large_lowd(3, n=20000), 3000, seed=1)]
    for inst in cases:
        u = np.rint(inst.points.astype(np.float64) * 1024)
        T = oracle.threshold(inst.eps)
        m = skc.DBSCAN(eps=math.sqrt(T + 0.5), min_samples=inst.min_pts).fit(u)
        lab, _, core = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
        sk_core = np.zeros(inst.n, bool)
        sk_core[m.core_sample_indices_] = True
        np.testing.assert_array_equal(core, sk_core)
        np.testing.assert_array_equal(lab == -1, m.labels_ == -1)
        # same partition of the core points
        pairs = {}
        for a, b in zip(lab[core], m.labels_[core]):
            assert pairs.setdefault(a, b) == b
        assert len(set(pairs.values())) == len(pairs)


def test_definition_by_transitive_closure_tiny():
    """Brute force on tiny inputs: Warshall's transitive closure of the core
    adjacency matrix (the plan discussed in Section VI) gives reachability;
    the labels must satisfy the cluster definition of Section II exactly."""
    rng = np.random.default_rng(21)
    for trial in range(300):
        n = int(rng.integers(1, 11))
        d = int(rng.integers(1, 4))
        x, u = _random_grid(rng, n, d, spread=8)
        eps = int(rng.integers(1, 5)) / 1024.0
        min_pts = int(rng.integers(1, 5))
        nb = neighbour_lists(x, eps)
        adj = np.zeros((n, n), bool)
        for i in range(n):
            adj[i, nb[i]] = True
        core = adj.sum(1) >= min_pts
        reach = adj & core[:, None] & core[None, :]
        for k in range(n):  # Warshall
            reach |= reach[:, k:k + 1] & reach[k:k + 1, :]
        lab, _, core_o = oracle.dbscan(x, eps, min_pts)
        np.testing.assert_array_equal(core_o, core)
        for p in range(n):
            if core[p]:
                members = [q for q in range(n) if core[q] and (reach[p, q] or q == p)]
                assert lab[p] == min(members)
            else:
                cn = [q for q in range(n) if core[q] and adj[p, q]]
                assert lab[p] == (lab[min(cn)] if cn else -1)


def test_permutation_gives_same_partition():
    inst = inputs.small_2d()
    lab, _, core = oracle.dbscan(inst.points, inst.eps, inst.min_pts)
    rng = np.random.default_rng(3)
    perm = rng.permutation(inst.n)
    lab_p, _, core_p = oracle.dbscan(inst.points[perm], inst.eps, inst.min_pts)
    back = np.empty_like(lab_p)
    back[perm] = lab_p
    core_back = np.empty_like(core_p)
    core_back[perm] = core_p
    np.testing.assert_array_equal(core_back, core)
    np.testing.assert_array_equal(back == -1, lab == -1)
    m = {}
    for a, b in zip(lab[core], back[core]):
        assert m.setdefault(a, b) == b
