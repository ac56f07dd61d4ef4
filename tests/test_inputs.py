"""The seeded generators: shapes, the 2^-10 grid, determinism, frozen eps."""
import numpy as np
import pytest

from paper_1506_02226_gb300 import inputs


def _on_grid(x):
    u = x.astype(np.float64) * 1024
    return np.all(u == np.floor(u)) and u.min() >= 0 and u.max() <= 1023


def test_small_2d_recipe():
    a, b = inputs.small_2d(), inputs.small_2d()
    assert a.points.shape == (2000, 2) and a.points.dtype == np.float32
    assert _on_grid(a.points) and np.array_equal(a.points, b.points)
    assert a.eps == float(np.float32(0.02)) and a.min_pts == 5


@pytest.mark.parametrize("d", [2, 3])
def test_large_lowd_recipe(d):
    inst = inputs.large_lowd(d, n=50_000)
    assert inst.points.shape == (50_000, d) and _on_grid(inst.points)
    assert inst.min_pts == 10 and inst.eps == float(np.float32(0.005))


def test_high_d_frozen_eps():
    assert inputs.derive_highd_eps() == inputs.HIGHD_EPS


def test_batch_and_serve_recipes():
    ns, ds = inputs.batch_sizes()
    assert len(ns) == 4096 and ns.min() >= 64 and ns.max() <= 8192
    assert set(np.unique(ds)) == {2, 3, 16}
    for inst in inputs.batch(count=8):
        assert _on_grid(inst.points) and 0.01 <= inst.eps <= 0.05 and 4 <= inst.min_pts <= 16
    job = inputs.serve_job(3)
    assert 1000 <= job.n <= 500_000 and job.d in (2, 3, 32) and _on_grid(job.points)
    t = inputs.serve_arrivals(100, 50.0)
    assert np.all(np.diff(t) > 0)


@pytest.mark.parametrize("d", [4, 8])
def test_mid_d_recipe(d):
    inst = inputs.mid_d(d, n=20_000)
    assert inst.points.shape == (20_000, d) and _on_grid(inst.points)
    assert inst.min_pts == 10 and inst.eps == float(np.float32(0.005 * np.sqrt(d / 2)))
    with pytest.raises(ValueError):
        inputs.mid_d(3)
