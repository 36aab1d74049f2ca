"""Parity at the full size of the headline workload (n = 90,000: 300x300 jittered grid,
theta0 = (1, 0.03, 1.0)), in the launch configuration bench.py times: covariance entries
sampled and checked one by one against the oracle, and properties of the mixed evaluation
that hold at any size (exact power-of-two scaling of sigma^2, bitwise repeatability)."""
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

M, THETA = 300, (1.0, 0.03, 1.0)


def test_fullsize_covariance_sampled_entries():
    import torch
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(M, 0)
    rng = np.random.default_rng(90)
    # 200 random locations plus a 10 x 10 patch of neighbouring grid points (short distances)
    r0, c0 = 137, 211
    patch = [(r0 + a) * M + c0 + b for a in range(10) for b in range(10)]
    idx = np.unique(np.concatenate([rng.choice(M * M, 200, replace=False), patch]))
    ref = np.tril(oracle.covariance(locs[idx], THETA))
    with exa.Context() as c:
        out = c.covariance(to_dev(locs), THETA)  # column-major lower triangle: (i, j) at out[j, i]
        it = torch.as_tensor(idx, device=out.device)
        T = out.index_select(0, it).index_select(1, it).cpu().numpy()
        del out
        torch.cuda.empty_cache()
    got = np.tril(T.T)
    d = locs[idx][:, None, :] - locs[idx][None, :, :]
    x = np.tril(np.sqrt((d ** 2).sum(-1))) / THETA[1]
    tol = (1e-13 + 4.4e-16 * x) * np.abs(ref) + 1e-300
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / (np.abs(ref) + 1e-300)))


def test_fullsize_mixed_scaling_and_repeatability():
    # sigma^2 = 4 scales every stored value by 4 and every factor entry by 2 exactly (all
    # splits and digit scales are powers of two), so log|Sigma| shifts by n ln 4 and the
    # quadratic form divides by 4, to rounding; the same call twice gives the same bits
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(M, 0)
    z = synth.normals(M * M, 7)
    dl, dz = to_dev(locs), to_dev(z)
    n = M * M
    with exa.Context() as c:
        a = c.loglik_ex(dl, dz, THETA, exa.EXA_MIXED_TF32X3)
        a2 = c.loglik_ex(dl, dz, THETA, exa.EXA_MIXED_TF32X3)
        b = c.loglik_ex(dl, dz, (4.0, THETA[1], THETA[2]), exa.EXA_MIXED_TF32X3)
    assert a["loglik"] == a2["loglik"] and a["logdet"] == a2["logdet"] and a["quad"] == a2["quad"]
    # (the refinement stops on the quadratic form, so the last residual may stay near 1e-4)
    assert a["n_tiles"] == 176 and 1 <= a["exact_band"] <= a["n_tiles"] and a["ir_resid"] <= 1e-3
    assert 0.0 < a["quad_err"] <= 1e-8
    assert abs(b["logdet"] - (a["logdet"] + n * math.log(4.0))) <= 1e-12 * abs(a["logdet"]) + 1e-9
    assert abs(b["quad"] - a["quad"] / 4.0) <= 1e-10 * a["quad"]
