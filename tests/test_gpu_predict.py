"""Kriging at new locations (Section IV's exact_predict) through the C ABI against the oracle:
means and variances element by element at sizes spanning several tiles with ragged tails,
interpolation at observed points, the variance blocks' ragged last block, and argument errors."""
import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1908_06936_gb300 as exa

    c = exa.Context()
    yield c
    c.close()


@pytest.mark.parametrize("m_obs,n_new,theta", [(9, 7, (1.0, 0.1, 0.5)), (23, 600, (1.5, 0.2, 1.5)),
                                               (17, 130, (0.8, 0.05, 1.0))])
def test_predict_vs_oracle(ctx, m_obs, n_new, theta):
    locs = synth.jittered_grid(m_obs, m_obs)
    z = oracle.simulate(locs, theta, synth.normals(m_obs * m_obs, m_obs))
    new = synth.uniform_square(n_new, m_obs + 1)
    mean_ref, var_ref = oracle.predict(locs, z, theta, new)
    mean, var = ctx.predict(to_dev(locs), to_dev(z), theta, to_dev(new))
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    scale = np.max(np.abs(z))
    assert np.all(np.abs(mean - mean_ref) <= 1e-9 * scale), np.max(np.abs(mean - mean_ref))
    assert np.all(np.abs(var - var_ref) <= 1e-9 * theta[0]), np.max(np.abs(var - var_ref))


def test_predict_interpolates_and_means_only(ctx):
    theta = (1.2, 0.1, 0.5)
    locs = synth.jittered_grid(20, 5)
    z = synth.normals(400, 5)
    idx = np.array([0, 1, 37, 200, 399])
    mean, var = ctx.predict(to_dev(locs), to_dev(z), theta, to_dev(locs[idx]))
    assert np.allclose(mean.cpu().numpy(), z[idx], rtol=0, atol=1e-9)
    assert np.all(np.abs(var.cpu().numpy()) <= 1e-9 * theta[0])
    m2, v2 = ctx.predict(to_dev(locs), to_dev(z), theta, to_dev(locs[idx]), variance=False)
    assert v2 is None and np.array_equal(m2.cpu().numpy(), mean.cpu().numpy())


def test_predict_arguments(ctx):
    import torch
    import paper_1908_06936_gb300 as exa

    locs = to_dev(synth.jittered_grid(4, 1))
    z = to_dev(synth.normals(16, 1))
    new = to_dev(synth.uniform_square(3, 2))
    mean = torch.empty(3, dtype=torch.float64, device="cuda")
    assert exa.exa_predict(ctx.handle, locs, z, (1.0, -0.1, 0.5), 16, new, 3, mean) == exa.EXA_ERR_ARG
    assert exa.exa_predict(ctx.handle, locs, z, (1.0, 0.1, 0.5), 16, new, 0, mean) == exa.EXA_OK
    bad = synth.jittered_grid(4, 1)
    bad[3, 0] = float("nan")  # a NaN location makes a pivot NaN
    assert exa.exa_predict(ctx.handle, to_dev(bad), z, (1.0, 0.1, 0.5), 16, new, 3, mean) == exa.EXA_ERR_NOT_SPD
