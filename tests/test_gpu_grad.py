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
    # the caller's precision is used for l and the gradient alike
    import paper_1908_06936_gb300 as exa

    th2 = torch.tensor([1.2, 0.12, 0.8], dtype=torch.float64, requires_grad=True)
    l2 = loglik(th2, to_dev(locs), to_dev(Z), ctx, prec=exa.EXA_MIXED_TF32X3)
    l2.backward()
    assert abs(l2.item() - ref["l"]) <= 1e-6 * abs(ref["l"])
    assert np.all(np.abs(th2.grad.numpy() - ref["grad"]) <= 5e-5 * max(1.0, np.max(np.abs(ref["grad"]))))


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


@pytest.mark.parametrize("m,cut,theta", [(40, 0, (1.0, 0.1, 0.5)), (24, 5, (1.5, 0.2, 1.5))])
def test_gradient_one_buffer_when_two_do_not_fit(m, cut, theta):
    # a context bound that holds the factor but not a second n x n buffer: Sigma^-1 is never
    # stored (X = L^-1 overwrites the factor, each tile of X^T X is reduced as it is formed);
    # the gradient still matches the oracle and the two-buffer path
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(m, seed=m + 1, theta0=theta)
    if cut:
        locs, Z = locs[:-cut], Z[:-cut]
    n = locs.shape[0]
    npad = -(-n // 128) * 128
    nn = npad * npad * 8
    ref = oracle.loglik_grad(locs, Z, theta)
    dl, dz = to_dev(locs), to_dev(Z)
    with exa.Context() as c2:
        l2, g2 = c2.loglik_grad(dl, dz, theta)
        held2 = exa.exa_workspace_bytes(c2.handle)  # the factor, Sigma^-1 and the small buffers
    assert held2 >= 2 * nn
    with exa.Context(workspace_bytes=held2 - nn // 2) as c1:  # everything but the second n x n buffer fits
        l1, g1 = c1.loglik_grad(dl, dz, theta)
        held1 = exa.exa_workspace_bytes(c1.handle)
    assert held1 < held2 - nn // 2  # no second n x n buffer (the gradient partials differ by a few KB)
    scale = max(1.0, float(np.max(np.abs(ref["grad"]))))
    assert abs(l1 - ref["l"]) <= 1e-10 * abs(ref["l"])
    assert np.all(np.abs(g1 - ref["grad"]) <= 1e-8 * scale), (g1, ref["grad"])
    assert np.all(np.abs(g1 - g2) <= 1e-10 * scale), (g1, g2)
    assert l1 == l2


def test_gradient_reuses_the_mixed_sigma_copy():
    # after a mixed-precision evaluation the context holds a second n x n buffer (the FP64 copy
    # of Sigma); the gradient takes it for Sigma^-1 instead of allocating a third
    import paper_1908_06936_gb300 as exa

    theta = (1.0, 0.1, 0.5)
    locs, Z = workload(40, seed=5, theta0=theta)
    dl, dz = to_dev(locs), to_dev(Z)
    ref = oracle.loglik_grad(locs, Z, theta)
    with exa.Context() as c:
        c.loglik(dl, dz, theta, exa.EXA_MIXED_TF32X3)
        before = exa.exa_workspace_bytes(c.handle)
        _, g = c.loglik_grad(dl, dz, theta)
        grown = exa.exa_workspace_bytes(c.handle) - before
    npad = -(-1600 // 128) * 128
    assert grown < npad * npad * 8
    scale = max(1.0, float(np.max(np.abs(ref["grad"]))))
    assert np.all(np.abs(g - ref["grad"]) <= 1e-8 * scale)


@pytest.mark.parametrize("m,theta", [(40, (1.0, 0.1, 0.5)), (50, (1.0, 0.03, 1.0)), (36, (1.5, 0.2, 1.5)),
                                     (60, (1.0, 0.1125, 1.0))])
def test_mixed_gradient_vs_oracle(ctx, m, theta):
    # mixed precision: l from the mixed evaluation, a = Sigma^-1 z refined in FP64, Sigma^-1 of the
    # mixed factor on the tensor cores (exact digit-slice products); stated bounds: l within
    # 1e-6 relative, each gradient component within 5e-5 of the largest.  The same factor with
    # Sigma^-1 on FP64 DMMA (exa_ctx_set_gradient_inverse) separates the factor's share of the error.
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(m, seed=m + 2, theta0=theta)
    ref = oracle.loglik_grad(locs, Z, theta)
    dl, dz = to_dev(locs), to_dev(Z)
    l, g = ctx.loglik_grad(dl, dz, theta, exa.EXA_MIXED_TF32X3)
    exa.exa_ctx_set_gradient_inverse(ctx.handle, 1)
    try:
        l64i, g64i = ctx.loglik_grad(dl, dz, theta, exa.EXA_MIXED_TF32X3)
    finally:
        exa.exa_ctx_set_gradient_inverse(ctx.handle, 0)
    scale = max(1.0, float(np.max(np.abs(ref["grad"]))))
    err = np.abs(g - ref["grad"]) / scale
    err64i = np.abs(g64i - ref["grad"]) / scale
    print("m=%d theta=%s |dl|/|l| %.2e grad err %s (FP64 inverse of the same factor: %s)"
          % (m, theta, abs(l - ref["l"]) / abs(ref["l"]), err, err64i))
    assert l64i == l
    assert abs(l - ref["l"]) <= 1e-6 * abs(ref["l"])
    assert np.all(err <= 5e-5), (g, ref["grad"])
    assert np.all(err64i <= 5e-5), (g64i, ref["grad"])


def test_mixed_gradient_ragged_and_repeatable(ctx):
    import paper_1908_06936_gb300 as exa

    theta = (1.0, 0.08, 0.8)
    locs, Z = workload(33, seed=9, theta0=theta)
    locs, Z = locs[:-7], Z[:-7]  # n = 1,082: three 512 blocks, the last one ragged
    dl, dz = to_dev(locs), to_dev(Z)
    ref = oracle.loglik_grad(locs, Z, theta)
    l1, g1 = ctx.loglik_grad(dl, dz, theta, exa.EXA_MIXED_TF32X3)
    l2, g2 = ctx.loglik_grad(dl, dz, theta, exa.EXA_MIXED_TF32X3)
    assert l1 == l2 and np.array_equal(g1, g2)
    scale = max(1.0, float(np.max(np.abs(ref["grad"]))))
    assert np.all(np.abs(g1 - ref["grad"]) <= 5e-5 * scale), (g1, ref["grad"])
    # the context still evaluates correctly afterwards (the factor buffer held X = L^-1)
    l3 = ctx.loglik(dl, dz, theta, exa.EXA_FP64)
    assert abs(l3 - ref["l"]) <= 1e-10 * abs(ref["l"])


def test_mixed_gradient_bf16_and_fp32_refused(ctx):
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(8, seed=1)
    for prec in (exa.EXA_MIXED_BF16X3, exa.EXA_MIXED_FP32):
        with pytest.raises(exa.ExaError) as ei:
            ctx.loglik_grad(to_dev(locs), to_dev(Z), (1.0, 0.1, 0.5), prec)
        assert ei.value.status == exa.EXA_ERR_ARG
