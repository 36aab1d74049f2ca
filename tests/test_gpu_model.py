"""Model options through the C ABI (nugget, great-circle distance) against the oracle with the
same options: covariance, FP64 and mixed log-likelihoods, gradient, prediction, Fisher and the
batched form."""
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


@pytest.fixture
def model(ctx):
    import paper_1908_06936_gb300 as exa

    def set_both(nugget, metric, radius):
        ctx.check(exa.exa_ctx_set_model(ctx.handle, nugget, metric, radius))
        oracle.set_model(nugget, metric, radius if radius > 0 else 6371.0)

    yield set_both
    exa.exa_ctx_set_model(ctx.handle, 0.0, 0, 0.0)
    oracle.set_model()


def lonlat(m, seed):
    g = synth.jittered_grid(m, seed)
    return np.ascontiguousarray(np.column_stack([-30.0 + 60.0 * g[:, 0], -20.0 + 40.0 * g[:, 1]]))


CASES = [(0.2, 0, 0.0, (1.0, 0.1, 0.5)), (0.0, 1, 0.0, (1.3, 800.0, 1.2)), (0.05, 1, 1.0, (0.9, 0.12, 0.7))]


@pytest.mark.parametrize("nugget,metric,radius,theta", CASES)
def test_covariance_and_loglik(ctx, model, nugget, metric, radius, theta):
    import torch
    import paper_1908_06936_gb300 as exa

    model(nugget, metric, radius)
    m = 21
    locs = lonlat(m, 4) if metric else synth.jittered_grid(m, 4)
    n = m * m
    z = oracle.simulate(locs, theta, synth.normals(n, 4))
    S = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    ctx.check(exa.exa_covariance(ctx.handle, to_dev(locs), n, theta, S, n))
    got = S.cpu().numpy().reshape(n, n).T  # column-major lower triangle
    ref = oracle.covariance(locs, theta)
    low = np.tril_indices(n)
    assert np.allclose(got[low], ref[low], rtol=1e-12, atol=1e-300)
    l_ref = oracle.loglik(locs, z, theta)["l"]
    l64 = ctx.loglik(to_dev(locs), to_dev(z), theta, exa.EXA_FP64)
    assert abs(l64 - l_ref) <= 1e-10 * abs(l_ref)
    lmx = ctx.loglik(to_dev(locs), to_dev(z), theta, exa.EXA_MIXED_TF32X3)
    assert abs(lmx - l_ref) <= 1e-6 * abs(l_ref)


@pytest.mark.parametrize("nugget,metric,radius,theta", CASES[:2])
def test_gradient_prediction_fisher(ctx, model, nugget, metric, radius, theta):
    model(nugget, metric, radius)
    m = 12
    locs = lonlat(m, 6) if metric else synth.jittered_grid(m, 6)
    z = oracle.simulate(locs, theta, synth.normals(m * m, 6))
    g_ref = oracle.loglik_grad(locs, z, theta)["grad"]
    _, g = ctx.loglik_grad(to_dev(locs), to_dev(z), theta)
    assert np.allclose(g, g_ref, rtol=1e-8, atol=1e-8 * np.max(np.abs(g_ref)))
    new = lonlat(5, 9)[:17] if metric else synth.uniform_square(17, 9)
    mean_ref, var_ref = oracle.predict(locs, z, theta, new)
    mean, var = ctx.predict(to_dev(locs), to_dev(z), theta, to_dev(new))
    assert np.allclose(mean.cpu().numpy(), mean_ref, rtol=0, atol=1e-9 * np.max(np.abs(z)))
    assert np.allclose(var.cpu().numpy(), var_ref, rtol=0, atol=1e-9 * theta[0])
    F_ref = oracle.fisher(locs, theta)
    F = ctx.fisher(to_dev(locs), theta)
    scale = np.sqrt(np.outer(np.diag(F_ref), np.diag(F_ref)))
    assert np.all(np.abs(F - F_ref) <= 1e-9 * scale)


def test_batched_with_model(ctx, model):
    import torch
    import paper_1908_06936_gb300 as exa

    model(0.1, 1, 0.0)
    sides = [6, 9, 13]
    theta = (1.0, 700.0, 0.8)
    locs = [lonlat(m, 20 + i) for i, m in enumerate(sides)]
    zs = [oracle.simulate(l, theta, synth.normals(l.shape[0], 20 + i)) for i, l in enumerate(locs)]
    ns = [l.shape[0] for l in locs]
    th = to_dev(np.tile(theta, 3))
    for prec, tol in ((exa.EXA_FP64, 1e-10), (exa.EXA_MIXED_FP32, 1e-6)):
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        st = torch.empty(3, dtype=torch.int32, device="cuda")
        ctx.check(exa.exa_loglik_batched(ctx.handle, 3, ns, [to_dev(l) for l in locs], [to_dev(z) for z in zs], th,
                                         prec, out, st))
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy() == 0)
        for r in range(3):
            ref = oracle.loglik(locs[r], zs[r], theta)["l"]
            assert abs(out[r].item() - ref) <= tol * abs(ref)


def test_model_arguments(ctx):
    import paper_1908_06936_gb300 as exa

    for args in ((-0.1, 0, 0.0), (0.0, 2, 0.0), (0.0, 1, -5.0), (float("nan"), 0, 0.0)):
        assert exa.exa_ctx_set_model(ctx.handle, *args) == exa.EXA_ERR_ARG
