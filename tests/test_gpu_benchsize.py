"""Parity against the FP64 oracle at n = 10,000 (100 x 100 jittered grid, theta = (1, 0.03, 1.0):
the short-range field of the headline workload, 20 panels of 512, so every phase of the mixed
schedule runs), in the launch configurations the benchmark times, plus the FP64 gradient at
n = 6,400.

Tolerances: FP64 log-likelihood |dl|/|l| <= 1e-10 (the FP64 bound); mixed precision
|dl|/|l| <= 1e-6 (the mixed bound) with the refined quadratic form within 1e-9 of the oracle's;
FP64 gradient within 1e-8 of the largest component.
"""
import numpy as np
import pytest

import oracle
from gpu_util import to_dev, workload

pytestmark = pytest.mark.gpu

M, THETA = 100, (1.0, 0.03, 1.0)


@pytest.fixture(scope="module")
def field():
    locs, z = workload(M, seed=21, theta0=THETA)  # Z = L eps, an exact realisation (oracle factor)
    ref = oracle.loglik(locs, z, THETA)
    assert ref["info"] == 0
    return locs, z, ref


@pytest.fixture(scope="module")
def ctx():
    import paper_1908_06936_gb300 as exa

    c = exa.Context()
    yield c
    c.close()


def test_fp64_n10000_vs_oracle(ctx, field):
    import paper_1908_06936_gb300 as exa

    locs, z, ref = field
    got = ctx.loglik_ex(to_dev(locs), to_dev(z), THETA, exa.EXA_FP64)
    assert abs(got["loglik"] - ref["l"]) <= 1e-10 * abs(ref["l"]), (got["loglik"], ref["l"])
    assert abs(got["logdet"] - ref["logdet"]) <= 1e-10 * abs(ref["logdet"])
    assert abs(got["quad"] - ref["quad"]) <= 1e-10 * abs(ref["quad"])


@pytest.mark.parametrize("mode", ["fused-pairs", "one-panel-single-cta", "default"])
def test_mixed_n10000_vs_oracle(ctx, field, mode):
    # fused-pairs: two panels per off-band pass forced for the whole factorisation (the bench's
    # phase above 61,440 rows) with far tiles on; one-panel-single-cta: the trailing update on
    # single CTAs (128 x 128 tiles), one panel at a time; default: the library's settings.
    import paper_1908_06936_gb300 as exa

    locs, z, ref = field
    if mode == "fused-pairs":
        exa.exa_ctx_set_panel_fusion(ctx.handle, 1)
    elif mode == "one-panel-single-cta":
        exa.exa_ctx_set_tc_pairs(ctx.handle, 0)
    try:
        got = ctx.loglik_ex(to_dev(locs), to_dev(z), THETA, exa.EXA_MIXED_TF32X3)
    finally:
        exa.exa_ctx_set_panel_fusion(ctx.handle, -1)
        exa.exa_ctx_set_tc_pairs(ctx.handle, 1)
    rel = abs(got["loglik"] - ref["l"]) / abs(ref["l"])
    print("%s: |dl|/|l| = %.3e, band %d of %d, %d refinement steps" % (mode, rel, got["exact_band"], got["n_tiles"],
                                                                      got["ir_iters"]))
    assert rel <= 1e-6
    assert abs(got["quad"] - ref["quad"]) <= 1e-9 * abs(ref["quad"])


def test_fp64_gradient_n6400_vs_oracle(ctx):
    theta = (1.5, 0.2, 1.5)  # the gradient configuration's theta on an 80 x 80 grid
    locs, z = workload(80, seed=22, theta0=theta)
    ref = oracle.loglik_grad(locs, z, theta)
    assert ref["info"] == 0
    l, g = ctx.loglik_grad(to_dev(locs), to_dev(z), theta)
    assert abs(l - ref["l"]) <= 1e-10 * abs(ref["l"])
    scale = max(1.0, float(np.max(np.abs(ref["grad"]))))
    assert np.all(np.abs(g - ref["grad"]) <= 1e-8 * scale), (g, ref["grad"])
