"""The seeded input recipes (shared by the oracle and the CUDA path's tests and benchmark) do what their
documentation states: jittered m x m grids on the unit square with the x index fastest, a minimum spacing of
0.2 / m, the seed streams, the theta perturbations and the replicate sizes."""
import numpy as np
import pytest

from paper_1908_06936_gb300 import synth


@pytest.mark.parametrize("m,seed", [(1, 0), (7, 3), (12, 0), (40, 5)])
def test_jittered_grid_cells_order_and_spacing(m, seed):
    s = synth.jittered_grid(m, seed)
    assert s.shape == (m * m, 2) and s.dtype == np.float64 and s.flags.c_contiguous
    assert np.all(s > 0.0) and np.all(s < 1.0)
    k = np.arange(m * m)
    ix, iy = k % m, k // m  # x index fastest
    off = s * m - np.stack([ix, iy], axis=1)  # position inside the cell, 0.5 +- 0.4
    assert np.all(np.abs(off - 0.5) <= 0.4 + 1e-12)
    if m > 1:
        d = np.sqrt(((s[:, None, :] - s[None, :, :]) ** 2).sum(-1))
        d[np.arange(m * m), np.arange(m * m)] = np.inf
        assert d.min() >= 0.2 / m - 1e-12
    assert np.array_equal(s, synth.jittered_grid(m, seed))
    if m > 1:
        assert not np.array_equal(s, synth.jittered_grid(m, seed + 1))


def test_seed_streams():
    assert np.array_equal(synth.normals(50, 4), np.random.default_rng(5).standard_normal(50))
    loc = np.random.default_rng(4).uniform(-0.4, 0.4, size=(9, 2))
    assert np.allclose(synth.jittered_grid(3, 4)[0], (0.5 + loc[0]) / 3)


def test_theta_perturbations_range_and_clipping():
    th0 = np.array([1.0, 0.1, 0.5])
    p = synth.theta_perturbations(th0, 200, seed=2)
    assert p.shape == (200, 3)
    assert np.all(p >= th0 * np.exp(-0.2) - 1e-15) and np.all(p <= th0 * np.exp(0.2) + 1e-15)
    assert np.array_equal(p, synth.theta_perturbations(th0, 200, seed=2))
    edge = synth.theta_perturbations([5.0, 0.01, 2.0], 100, seed=1)  # at the bounds: clipped into them
    assert np.all(edge >= synth.THETA_LOWER) and np.all(edge <= synth.THETA_UPPER)
    assert edge[:, 0].max() == 5.0 and edge[:, 1].min() == 0.01 and edge[:, 2].max() == 2.0


def test_replicate_sides_and_uniform_square():
    m = synth.replicate_sides(256, seed=5)
    assert m.shape == (256,) and m.min() >= 20 and m.max() <= 80 and np.issubdtype(m.dtype, np.integer)
    assert np.array_equal(m, synth.replicate_sides(256, seed=5))
    u = synth.uniform_square(1000, seed=3)
    assert u.shape == (1000, 2) and np.all(u >= 0.0) and np.all(u < 1.0)
