"""Parity of the FP64 CUDA path (steps a1-a5) with the FP64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from gpu_util import lower_colmajor, to_dev, workload

pytestmark = pytest.mark.gpu

def matern_tol(locs, theta, ref):
    """1e-13 relative, plus the conditioning of exp(-x): one ulp of x = r/beta is 2.2e-16 x relative."""
    d = locs[:, None, :] - locs[None, :, :]
    x = np.tril(np.sqrt((d ** 2).sum(-1))) / theta[1]
    return (1e-13 + 4.4e-16 * x) * np.abs(ref) + 1e-300


THETAS = [(1.0, 0.1, 0.5), (1.0, 0.03, 1.0), (1.5, 0.2, 1.5), (0.7, 0.05, 0.25), (2.0, 0.3, 2.0),
          (1.2, 0.08, 0.73), (1.0, 0.1, 1.999999), (0.4, 0.5, 0.1)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_1908_06936_gb300 as exa

    assert torch.cuda.is_available()
    c = exa.Context()
    yield c
    c.close()


@pytest.mark.parametrize("m,ragged", [(40, 0), (9, 0), (13, 5), (24, 1)])
@pytest.mark.parametrize("theta", THETAS)
def test_covariance_elementwise(ctx, m, ragged, theta):
    locs = synth.jittered_grid(m, seed=m)
    if ragged:
        locs = locs[:-ragged]
    n = locs.shape[0]
    ref = np.tril(oracle.covariance(locs, theta))
    got = lower_colmajor(ctx.covariance(to_dev(locs), theta), n)
    err = np.abs(got - ref)
    assert np.all(err <= matern_tol(locs, theta, ref)), (float(np.max(err / (np.abs(ref) + 1e-300))), theta)


def test_covariance_extreme_distances(ctx):
    # coincident points, tiny and huge separations (x up to 1e5: exact underflow to 0)
    locs = np.array([[0.0, 0.0], [0.0, 0.0], [1e-9, 0.0], [0.3, 0.4], [50.0, 0.0], [1e3, 1e3]])
    for theta in [(1.0, 0.1, 0.5), (2.0, 0.03, 1.0), (1.0, 0.01, 1.3)]:
        ref = np.tril(oracle.covariance(locs, theta))
        got = lower_colmajor(ctx.covariance(to_dev(locs), theta), 6)
        assert np.all(np.abs(got - ref) <= matern_tol(locs, theta, ref))


@pytest.mark.parametrize("m,ragged", [(40, 0), (12, 3), (16, 0)])
@pytest.mark.parametrize("theta", THETAS[:4])
def test_potrf_factor(ctx, m, ragged, theta):
    import paper_1908_06936_gb300 as exa
    import torch

    locs = synth.jittered_grid(m, seed=100 + m)
    if ragged:
        locs = locs[:-ragged]
    n = locs.shape[0]
    S = oracle.covariance(locs, theta)
    Lref, info = oracle.cholesky(S)
    assert info == 0
    # column-major buffer: pass S^T (== S), read back transposed
    a = torch.as_tensor(S.copy(), device="cuda")
    ctx.check(exa.exa_potrf(ctx.handle, a, n, n))
    L = np.tril(a.cpu().numpy().T)
    scale = np.max(np.abs(Lref))
    assert np.max(np.abs(L - Lref)) <= 1e-10 * scale
    # strict upper triangle of the caller's matrix is untouched
    assert np.array_equal(np.triu(a.cpu().numpy().T, 1), np.triu(S, 1))


@pytest.mark.parametrize("tile_nb", [64, 128])
def test_loglik_config1_theta0_and_perturbations(tile_nb):
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(40, seed=0)
    dl, dz = to_dev(locs), to_dev(Z)
    thetas = [(1.0, 0.1, 0.5)] + [tuple(t) for t in synth.theta_perturbations((1.0, 0.1, 0.5), 10, seed=0)]
    with exa.Context(tile_nb=tile_nb) as c:
        for th in thetas:
            ref = oracle.loglik(locs, Z, th)
            got = c.loglik_ex(dl, dz, th)
            assert abs(got["loglik"] - ref["l"]) <= 1e-10 * abs(ref["l"]), (th, got["loglik"], ref["l"])
            assert abs(got["logdet"] - ref["logdet"]) <= 1e-10 * abs(ref["logdet"]) + 1e-9
            assert abs(got["quad"] - ref["quad"]) <= 1e-10 * abs(ref["quad"])


@pytest.mark.parametrize("m,ragged,theta", [(7, 0, (1.0, 0.1, 0.5)), (13, 2, (1.5, 0.2, 1.5)),
                                            (23, 7, (1.0, 0.03, 1.0)), (1, 0, (2.0, 0.1, 0.5)),
                                            (2, 2, (1.0, 0.1, 0.5)), (30, 0, (0.7, 0.05, 0.25))])
def test_loglik_ragged_and_tiny(ctx, m, ragged, theta):
    locs = synth.jittered_grid(m, seed=7 * m)
    Z = synth.normals(m * m, seed=m)
    if ragged:
        locs, Z = locs[:-ragged] if ragged < m * m else locs[:1], Z[:-ragged] if ragged < m * m else Z[:1]
    ref = oracle.loglik(locs, Z, theta)
    got = ctx.loglik_ex(to_dev(locs), to_dev(Z), theta)
    assert abs(got["loglik"] - ref["l"]) <= 1e-10 * abs(ref["l"])


def test_loglik_n1_closed_form(ctx):
    z = -0.8
    got = ctx.loglik(to_dev(np.array([[0.2, 0.7]])), to_dev(np.array([z])), (2.5, 0.1, 0.5))
    ref = -0.5 * math.log(2 * math.pi) - 0.5 * math.log(2.5) - z * z / 5.0
    assert abs(got - ref) <= 1e-14 * abs(ref)


def test_loglik_deterministic(ctx):
    locs, Z = workload(40, seed=0)
    dl, dz = to_dev(locs), to_dev(Z)
    a = ctx.loglik_ex(dl, dz, (1.0, 0.1, 0.5))
    b = ctx.loglik_ex(dl, dz, (1.0, 0.1, 0.5))
    assert a["loglik"] == b["loglik"] and a["logdet"] == b["logdet"] and a["quad"] == b["quad"]


def test_loglik_independence_limit(ctx):
    locs = synth.jittered_grid(40, seed=3)
    Z = synth.normals(1600, 3)
    s2 = 1.7
    got = ctx.loglik(to_dev(locs), to_dev(Z), (s2, 1e-4, 1.0))
    ref = -800 * math.log(2 * math.pi * s2) - float(Z @ Z) / (2 * s2)
    assert abs(got - ref) <= 1e-13 * abs(ref)


def test_not_spd_reports_pivot(ctx):
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(20, seed=1)
    locs[217, 1] = float("nan")
    with pytest.raises(exa.ExaError) as ei:
        ctx.loglik(to_dev(locs), to_dev(synth.normals(400, 1)), (1.0, 0.1, 0.5))
    assert ei.value.status == exa.EXA_ERR_NOT_SPD
    assert ei.value.pivot == 217
    # the context stays usable
    locs2, Z2 = workload(9, seed=2)
    assert math.isfinite(ctx.loglik(to_dev(locs2), to_dev(Z2), (1.0, 0.1, 0.5)))


def test_bad_arguments(ctx):
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(5, seed=4)
    for th in [(0.0, 0.1, 0.5), (1.0, -0.1, 0.5), (1.0, 0.1, float("nan")), (1.0, float("inf"), 1.0)]:
        with pytest.raises(exa.ExaError) as ei:
            ctx.loglik(to_dev(locs), to_dev(Z), th)
        assert ei.value.status == exa.EXA_ERR_ARG


def test_simulate_matches_oracle(ctx):
    locs = synth.jittered_grid(20, seed=5)
    eps = synth.normals(400, 5)
    th = (1.0, 0.1, 0.5)
    ref = oracle.simulate(locs, th, eps)
    got = ctx.simulate(to_dev(locs), to_dev(eps), th).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_workspace_limit_reports_nomem():
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(20, seed=6)
    with exa.Context(workspace_bytes=1 << 20) as c:
        with pytest.raises(exa.ExaError) as ei:
            c.loglik(to_dev(locs), to_dev(Z), (1.0, 0.1, 0.5))
        assert ei.value.status == exa.EXA_ERR_NOMEM


@pytest.mark.parametrize("theta", [(1.0, 0.03, 1.0), (1.0, 0.1, 0.5), (2.0, 0.2, 1.5), (0.7, 0.05, 0.27),
                                   (1.0, 0.1, 1.999999), (1.0, 1.0, 0.1)])
def test_covariance_dense_distances(ctx, theta):
    # points on a line at geometric offsets: x = r / beta sweeps 1e-3 .. 900 across every
    # table segment boundary (octaves and eighths) and the exact-routine cut-off
    xs = np.concatenate([[0.0], np.geomspace(1e-3, 900.0, 700) * theta[1]])
    locs = np.stack([xs, np.zeros_like(xs)], axis=1)
    ref = np.tril(oracle.covariance(locs, theta))
    got = lower_colmajor(ctx.covariance(to_dev(locs), theta), locs.shape[0])
    err = np.abs(got - ref)
    assert np.all(err <= matern_tol(locs, theta, ref)), float(np.max(err / (np.abs(ref) + 1e-300)))
