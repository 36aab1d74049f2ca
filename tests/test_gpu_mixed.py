"""Mixed-precision path (MP variant of Section II-A, Fig. 1(d)) against the FP64 oracle.

Stated bound: |dl|/|l| <= 1e-6 (the accuracy the mixed form must keep); the
quadratic form is refined in FP64 to a relative residual below 1e-11.
"""
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


@pytest.mark.parametrize("m,theta", [(40, (1.0, 0.1, 0.5)), (50, (1.0, 0.18, 1.0)), (80, (1.0, 0.1125, 1.0)),
                                     (37, (1.5, 0.2, 1.5)), (60, (1.0, 0.03, 1.0))])
def test_mixed_vs_oracle(ctx, m, theta):
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(m, seed=m, theta0=theta)
    ref = oracle.loglik(locs, Z, theta)
    got = ctx.loglik_ex(to_dev(locs), to_dev(Z), theta, exa.EXA_MIXED_TF32X3)
    rel = abs(got["loglik"] - ref["l"]) / abs(ref["l"])
    print("m=%d theta=%s |dl|/|l|=%.3e ir_iters=%d ir_resid=%.2e" % (m, theta, rel, got["ir_iters"], got["ir_resid"]))
    assert rel <= 1e-6
    # the refinement stops once q is final (its variational estimate is second order in the
    # residual), so the last residual taken may stay near 1e-4; q itself is checked below
    assert got["ir_resid"] <= 1e-3
    assert 1 <= got["exact_band"] <= got["n_tiles"]
    # the refined quadratic form is accurate far beyond the factor's precision
    assert abs(got["quad"] - ref["quad"]) <= 1e-9 * abs(ref["quad"])


def test_mixed_matches_gpu_fp64(ctx):
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(64, seed=3, theta0=(1.0, 0.1, 0.5))
    dl, dz = to_dev(locs), to_dev(Z)
    for th in [(1.0, 0.1, 0.5), (0.8, 0.07, 0.9)]:
        f = ctx.loglik_ex(dl, dz, th, exa.EXA_FP64)
        mx = ctx.loglik_ex(dl, dz, th, exa.EXA_MIXED_TF32X3)
        assert abs(mx["loglik"] - f["loglik"]) <= 1e-6 * abs(f["loglik"])


def test_mixed_power_of_two_scaling_is_exact(ctx):
    # sigma^2 = 4 scales every stored value by 4 and every factor entry by 2 exactly, so
    # log|Sigma| shifts by n ln 4 and the quadratic form divides by 4, both to rounding
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(48, seed=4, theta0=(1.0, 0.1, 1.0))
    dl, dz = to_dev(locs), to_dev(Z)
    n = locs.shape[0]
    a = ctx.loglik_ex(dl, dz, (1.0, 0.1, 1.0), exa.EXA_MIXED_TF32X3)
    b = ctx.loglik_ex(dl, dz, (4.0, 0.1, 1.0), exa.EXA_MIXED_TF32X3)
    assert abs(b["logdet"] - (a["logdet"] + n * math.log(4.0))) <= 1e-12 * abs(a["logdet"]) + 1e-9
    assert abs(b["quad"] - a["quad"] / 4.0) <= 1e-11 * a["quad"]


def test_mixed_independence_limit(ctx):
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(40, seed=3)
    Z = synth.normals(1600, 3)
    s2 = 1.7
    got = ctx.loglik(to_dev(locs), to_dev(Z), (s2, 1e-4, 1.0), exa.EXA_MIXED_TF32X3)
    ref = -800 * math.log(2 * math.pi * s2) - float(Z @ Z) / (2 * s2)
    assert abs(got - ref) <= 1e-13 * abs(ref)


def test_mixed_tiny_and_ragged(ctx):
    import paper_1908_06936_gb300 as exa

    for m, cut in [(1, 0), (5, 3), (16, 1), (17, 0)]:
        locs = synth.jittered_grid(m, seed=m)[: m * m - cut]
        Z = synth.normals(m * m, seed=m)[: m * m - cut]
        ref = oracle.loglik(locs, Z, (1.0, 0.1, 0.5))["l"]
        got = ctx.loglik(to_dev(locs), to_dev(Z), (1.0, 0.1, 0.5), exa.EXA_MIXED_TF32X3)
        assert abs(got - ref) <= 1e-6 * abs(ref)


def test_mixed_not_spd(ctx):
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(30, seed=1)
    locs[611, 0] = float("nan")
    with pytest.raises(exa.ExaError) as ei:
        ctx.loglik(to_dev(locs), to_dev(synth.normals(900, 1)), (1.0, 0.1, 0.5), exa.EXA_MIXED_TF32X3)
    assert ei.value.status == exa.EXA_ERR_NOT_SPD


def test_bf16x3_is_refused_with_reason(ctx):
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(8, seed=1)
    with pytest.raises(exa.ExaError) as ei:
        ctx.loglik(to_dev(locs), to_dev(Z), (1.0, 0.1, 0.5), exa.EXA_MIXED_BF16X3)
    assert ei.value.status == exa.EXA_ERR_ARG and "3e-4" in str(ei.value)


def test_precision_enum_values_and_fp32_refusal(ctx):
    """The precision codes are the boundary's (FP64 0, FP32 1, BF16x3 2, TF32x3 3); the single-field
    path refuses EXA_MIXED_FP32 (batched form only) with its reason."""
    import paper_1908_06936_gb300 as exa

    assert (exa.EXA_FP64, exa.EXA_MIXED_FP32, exa.EXA_MIXED_BF16X3, exa.EXA_MIXED_TF32X3) == (0, 1, 2, 3)
    locs, Z = workload(8, seed=1)
    with pytest.raises(exa.ExaError) as ei:
        ctx.loglik(to_dev(locs), to_dev(Z), (1.0, 0.1, 0.5), exa.EXA_MIXED_FP32)
    assert ei.value.status == exa.EXA_ERR_ARG and "batched" in str(ei.value)


def test_mixed_simulate_close_to_oracle(ctx):
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(20, seed=5)
    eps = synth.normals(400, 5)
    th = (1.0, 0.1, 0.5)
    ref = oracle.simulate(locs, th, eps)
    got = ctx.simulate(to_dev(locs), to_dev(eps), th, exa.EXA_MIXED_TF32X3).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_mixed_all_exact_is_fp64_grade(ctx):
    # every tile through the exact digit-slice products: error far below the TF32x3 tiles
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(37, seed=37, theta0=(1.5, 0.2, 1.5))
    ref = oracle.loglik(locs, Z, (1.5, 0.2, 1.5))
    exa.exa_ctx_set_mixed_band(ctx.handle, -1)
    try:
        got = ctx.loglik_ex(to_dev(locs), to_dev(Z), (1.5, 0.2, 1.5), exa.EXA_MIXED_TF32X3)
    finally:
        exa.exa_ctx_set_mixed_band(ctx.handle, 0)
    assert got["exact_band"] == got["n_tiles"]
    assert abs(got["loglik"] - ref["l"]) <= 1e-8 * abs(ref["l"])


def test_mixed_ill_conditioned_reports_nonconvergence_or_is_accurate(ctx):
    # a very smooth, long-range field: either the refinement converges (and l is accurate)
    # or the library says it did not; it never returns a silently wrong value
    import paper_1908_06936_gb300 as exa

    m, th = 60, (1.5, 0.2, 1.5)
    locs, Z = workload(m, seed=2, theta0=th)
    ref = oracle.loglik(locs, Z, th)
    try:
        got = ctx.loglik_ex(to_dev(locs), to_dev(Z), th, exa.EXA_MIXED_TF32X3)
    except exa.ExaError as e:
        assert e.status == exa.EXA_ERR_IR_NOCONV
        return
    assert abs(got["loglik"] - ref["l"]) <= 1e-6 * abs(ref["l"])


def test_mixed_pair_and_single_cta_updates_agree(ctx):
    # the off-band trailing update on CTA pairs and on single CTAs accumulate the same
    # products in the same order per tile: the log-likelihoods agree to rounding
    import paper_1908_06936_gb300 as exa

    theta = (1.0, 0.05, 1.0)
    locs, Z = workload(72, seed=72, theta0=theta)
    dl, dz = to_dev(locs), to_dev(Z)
    exa.exa_ctx_set_far_tile_margin(ctx.handle, 0)  # every off-band tile with three products
    exa.exa_ctx_set_tc_pairs(ctx.handle, 0)
    try:
        single = ctx.loglik_ex(dl, dz, theta, exa.EXA_MIXED_TF32X3)
        exa.exa_ctx_set_tc_pairs(ctx.handle, 1)
        pair = ctx.loglik_ex(dl, dz, theta, exa.EXA_MIXED_TF32X3)
    finally:
        exa.exa_ctx_set_tc_pairs(ctx.handle, 1)
        exa.exa_ctx_set_far_tile_margin(ctx.handle, 16)
    assert abs(pair["loglik"] - single["loglik"]) <= 1e-12 * abs(single["loglik"])
    ref = oracle.loglik(locs, Z, theta)["l"]
    assert abs(pair["loglik"] - ref) <= 1e-6 * abs(ref)


def test_far_tiles_single_product_keeps_accuracy(ctx):
    # with a short correlation length most of the trailing matrix is far from the diagonal and its
    # panel blocks are tiny: those tiles take one TF32 product.  The result must stay within the
    # mixed bound of the FP64 evaluation and close to the all-three-product result.
    import paper_1908_06936_gb300 as exa

    theta = (1.0, 0.03, 1.0)
    m = 100
    locs = synth.jittered_grid(m, 11)
    z = synth.normals(m * m, 11)
    dl, dz = to_dev(locs), to_dev(z)
    l64 = ctx.loglik(dl, dz, theta, exa.EXA_FP64)
    far = ctx.loglik_ex(dl, dz, theta, exa.EXA_MIXED_TF32X3)["loglik"]
    exa.exa_ctx_set_far_tile_margin(ctx.handle, 0)
    try:
        three = ctx.loglik_ex(dl, dz, theta, exa.EXA_MIXED_TF32X3)["loglik"]
    finally:
        exa.exa_ctx_set_far_tile_margin(ctx.handle, 16)
    print("far %.3e three %.3e" % (abs(far - l64) / abs(l64), abs(three - l64) / abs(l64)))
    assert abs(far - l64) <= 1e-6 * abs(l64)
    assert abs(far - three) <= 1e-7 * abs(l64)


@pytest.mark.parametrize("m,theta,min_rows", [(50, (1.0, 0.1, 0.5), 1), (72, (1.0, 0.05, 1.0), 1),
                                              (100, (1.0, 0.03, 1.0), 1), (100, (1.0, 0.03, 1.0), 4096),
                                              (64, (1.5, 0.2, 1.5), 1)])
def test_two_panel_passes_match_one_panel_order(ctx, m, theta, min_rows):
    # panels applied in pairs (one K = 1024 TF32x3 pass per pair off the band, the side
    # stream factoring two panels ahead) and one at a time differ only in the rounding of
    # the FP32 partial sums.  n = 2,500 has five panels (one pair, then the hand-over);
    # min_rows = 4096 at n = 10,000 switches to the one-panel order midway.
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(m, m + 1)
    dl, dz = to_dev(locs), to_dev(synth.normals(m * m, m + 1))
    exa.exa_ctx_set_panel_fusion(ctx.handle, min_rows)
    try:
        fused = ctx.loglik_ex(dl, dz, theta, exa.EXA_MIXED_TF32X3)
        exa.exa_ctx_set_panel_fusion(ctx.handle, 0)
        single = ctx.loglik_ex(dl, dz, theta, exa.EXA_MIXED_TF32X3)
    finally:
        exa.exa_ctx_set_panel_fusion(ctx.handle, -1)
    l64 = ctx.loglik(dl, dz, theta, exa.EXA_FP64)
    print("fused %.3e one-panel %.3e" % (abs(fused["loglik"] - l64) / abs(l64), abs(single["loglik"] - l64) / abs(l64)))
    assert abs(fused["loglik"] - l64) <= 1e-6 * abs(l64)
    assert abs(fused["loglik"] - single["loglik"]) <= 1e-7 * abs(l64)
    assert fused["exact_band"] == single["exact_band"]


def test_panel_fusion_setting(ctx):
    import paper_1908_06936_gb300 as exa

    assert exa.exa_ctx_set_panel_fusion(ctx.handle, 12345) == exa.EXA_OK
    assert exa.exa_ctx_set_panel_fusion(ctx.handle, -7) == exa.EXA_OK
    assert exa.exa_ctx_set_panel_fusion(0, 1) == exa.EXA_ERR_ARG


def test_refinement_to_residual_target(ctx):
    # with a residual target the refinement continues past the quadratic-form rule: the relative
    # residual ||z - Sigma x|| / ||z|| reaches 1e-14 (the refinement pin), and l is unchanged to
    # well within the mixed bound
    import paper_1908_06936_gb300 as exa

    theta = (1.0, 0.1, 0.5)
    locs, Z = workload(40, seed=12, theta0=theta)
    dl, dz = to_dev(locs), to_dev(Z)
    ref = oracle.loglik(locs, Z, theta)
    a = ctx.loglik_ex(dl, dz, theta, exa.EXA_MIXED_TF32X3)
    assert exa.exa_ctx_set_refinement(ctx.handle, 1e-14) == exa.EXA_OK
    try:
        b = ctx.loglik_ex(dl, dz, theta, exa.EXA_MIXED_TF32X3)
    finally:
        exa.exa_ctx_set_refinement(ctx.handle, 0.0)
    print("default: %d steps, resid %.2e; target 1e-14: %d steps, resid %.2e" % (a["ir_iters"], a["ir_resid"],
                                                                               b["ir_iters"], b["ir_resid"]))
    assert b["ir_resid"] <= 1e-14
    assert b["ir_iters"] >= a["ir_iters"]
    assert abs(b["quad"] - ref["quad"]) <= 1e-12 * abs(ref["quad"])
    assert abs(b["loglik"] - ref["l"]) <= 1e-6 * abs(ref["l"])
    assert exa.exa_ctx_set_refinement(ctx.handle, -1.0) == exa.EXA_ERR_ARG
    for bad in (-1e-9, 1e-3, float("nan")):
        assert exa.exa_ctx_set_refinement_quad(ctx.handle, bad) == exa.EXA_ERR_ARG
    # the default rule's q (the variational estimate, when it ends the refinement) agrees with the
    # q of a solution refined to rounding level within its reported error estimate, and with the
    # oracle's
    assert 0.0 < a["quad_err"] <= 1e-8
    assert abs(a["quad"] - b["quad"]) <= a["quad_err"] * abs(b["quad"]) + 1e-12 * abs(b["quad"])
    assert abs(a["quad"] - ref["quad"]) <= 1e-9 * abs(ref["quad"])


@pytest.mark.parametrize("theta", [(1.0, 0.03, 0.5), (1.0, 0.1, 1.0), (1.0, 0.3, 0.5), (2.0, 0.05, 1.5)])
def test_quadratic_form_stopping_rule_vs_oracle(ctx, theta):
    # short- and long-range, rough and smooth fields on a 70 x 70 grid (ten 512 panels): the
    # quadratic form of the default stopping rule against the oracle's (to 1e-9) and against the
    # same factor's solution refined to rounding level (within the reported error estimate)
    import paper_1908_06936_gb300 as exa

    locs, Z = workload(70, seed=31, theta0=theta)
    ref = oracle.loglik(locs, Z, theta)
    got = ctx.loglik_ex(to_dev(locs), to_dev(Z), theta, exa.EXA_MIXED_TF32X3)
    print("theta %s: %d refinement steps, resid %.2e, |dq|/|q| %.2e" % (
        theta, got["ir_iters"], got["ir_resid"], abs(got["quad"] - ref["quad"]) / abs(ref["quad"])))
    assert abs(got["quad"] - ref["quad"]) <= 1e-9 * abs(ref["quad"])
    assert abs(got["loglik"] - ref["l"]) <= 1e-6 * abs(ref["l"])
    # against the same factor's solution refined to rounding level (no oracle rounding involved):
    # within the error estimate the call reports, itself within the 1e-8 default
    assert exa.exa_ctx_set_refinement(ctx.handle, 1e-14) == exa.EXA_OK
    try:
        tight = ctx.loglik_ex(to_dev(locs), to_dev(Z), theta, exa.EXA_MIXED_TF32X3)
    finally:
        exa.exa_ctx_set_refinement(ctx.handle, 0.0)
    assert got["quad_err"] <= 1e-8
    assert abs(got["quad"] - tight["quad"]) <= got["quad_err"] * abs(tight["quad"]) + 1e-12 * abs(tight["quad"])
