"""Gradient path (hand-written adjoint) against the FP64 oracle, closed forms and finite differences."""
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from gpu_util import to_dev, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1908_06936_gb300 as exa

    c = exa.Context()
    yield c
    c.close()


@pytest.mark.parametrize("m,cut,theta", [(20, 0, (1.5, 0.2, 1.5)), (24, 5, (1.0, 0.1, 0.5)),
                                         (30, 0, (0.8, 0.05, 1.0)), (13, 0, (2.0, 0.3, 0.73)),
                                         (40, 0, (1.0, 0.1, 0.5))])
def test_gradient_vs_oracle(ctx, m, cut, theta):
    locs, Z = workload(m, seed=m, theta0=theta)
    if cut:
        locs, Z = locs[:-cut], Z[:-cut]
    ref = oracle.loglik_grad(locs, Z, theta)
    l, g = ctx.loglik_grad(to_dev(locs), to_dev(Z), theta)
    assert abs(l - ref["l"]) <= 1e-10 * abs(ref["l"])
    scale = max(1.0, float(np.max(np.abs(ref["grad"]))))
    assert np.all(np.abs(g - ref["grad"]) <= 1e-8 * scale), (g, ref["grad"])


def test_gradient_sigma2_closed_form(ctx):
    # Sigma is proportional to sigma^2: dl/dsigma^2 = (z^T Sigma^-1 z - n) / (2 sigma^2)
    locs, Z = workload(36, seed=3, theta0=(1.0, 0.1, 1.0))
    for s2 in [0.6, 1.0, 2.5]:
        th = (s2, 0.1, 1.0)
        r = ctx.loglik_ex(to_dev(locs), to_dev(Z), th)
        _, g = ctx.loglik_grad(to_dev(locs), to_dev(Z), th)
        ref = (r["quad"] - locs.shape[0]) / (2 * s2)
        assert abs(g[0] - ref) <= 1e-10 * max(1.0, abs(ref)) * locs.shape[0]


def test_gradient_central_differences(ctx):
    # config-4 check: central differences with h = 1e-6 relative, |g - g_FD| / |g|_inf <= 1e-5
    theta = (1.5, 0.2, 1.5)
    locs, Z = workload(40, seed=4, theta0=theta)
    dl, dz = to_dev(locs), to_dev(Z)
    _, g = ctx.loglik_grad(dl, dz, theta)
    fd = np.zeros(3)
    for k in range(3):
        h = 1e-6 * theta[k]
        tp = list(theta); tp[k] += h
        tm = list(theta); tm[k] -= h
        fd[k] = (ctx.loglik(dl, dz, tp) - ctx.loglik(dl, dz, tm)) / (2 * h)
    assert np.max(np.abs(g - fd)) / np.max(np.abs(g)) <= 1e-5, (g, fd)


def test_gradient_tile64_and_zero_at_profile_sigma2():
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(21, seed=6, theta0=(1.0, 0.1, 0.5))
    with exa.Context(tile_nb=64) as c:
        r = c.loglik_ex(to_dev(locs), to_dev(Z), (1.0, 0.1, 0.5))
        s2hat = r["quad"] / locs.shape[0]
        _, g = c.loglik_grad(to_dev(locs), to_dev(Z), (s2hat, 0.1, 0.5))
    assert abs(g[0]) <= 1e-9 * locs.shape[0] / s2hat


def test_autograd_function(ctx):
    import torch
    from paper_1908_06936_gb300.autograd import loglik

    locs, Z = workload(16, seed=8, theta0=(1.0, 0.1, 0.5))
    th = torch.tensor([1.2, 0.12, 0.8], dtype=torch.float64, requires_grad=True)
    l = loglik(th, to_dev(locs), to_dev(Z), ctx)
    (2.0 * l).backward()
    ref = oracle.loglik_grad(locs, Z, (1.2, 0.12, 0.8))
    assert abs(l.item() - ref["l"]) <= 1e-10 * abs(ref["l"])
    assert np.allclose(th.grad.numpy(), 2.0 * ref["grad"], rtol=1e-8, atol=1e-8)


def test_gradient_not_spd(ctx):
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(12, seed=1)
    locs[40, 0] = float("nan")
    with pytest.raises(exa.ExaError) as ei:
        ctx.loglik_grad(to_dev(locs), to_dev(synth.normals(144, 1)), (1.0, 0.1, 0.5))
    assert ei.value.status == exa.EXA_ERR_NOT_SPD


def test_mle_drivers_agree(ctx):
    # both drivers maximise the same l through the library; the gradient driver must reach
    # at least the derivative-free optimum
    from paper_1908_06936_gb300 import mle

    locs, Z = workload(20, seed=11, theta0=(1.0, 0.1, 0.5))
    dl, dz = to_dev(locs), to_dev(Z)
    a = mle.fit_derivative_free(dl, dz, maxfev=150, ctx=ctx)
    b = mle.fit_gradient(dl, dz, x0=[0.5, 0.05, 0.3], ctx=ctx)
    assert b["loglik"] >= a["loglik"] - 1e-3
    assert math.isfinite(a["loglik"])
