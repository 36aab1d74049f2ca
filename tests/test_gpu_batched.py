"""Batched replicate fields (one persistent launch) against the FP64 oracle, plus failure paths."""
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def make_batch(sides, seed, theta0=(1.0, 0.1, 0.5), with_z=True):
    locs, zs = [], []
    for r, m in enumerate(sides):
        l = synth.jittered_grid(int(m), seed + r)
        locs.append(l)
        zs.append(oracle.simulate(l, theta0, synth.normals(int(m) ** 2, seed + r)) if with_z
                  else synth.normals(int(m) ** 2, seed + r))
    return locs, zs


def run(ctx, locs, zs, thetas, prec=0):
    import torch
    import paper_1908_06936_gb300 as exa

    ns = [l.shape[0] for l in locs]
    dl = [to_dev(l) for l in locs]
    dz = [to_dev(z) for z in zs]
    th = to_dev(np.asarray(thetas, dtype=np.float64).ravel())
    out = torch.empty(len(ns), dtype=torch.float64, device="cuda")
    st = torch.empty(len(ns), dtype=torch.int32, device="cuda")
    ctx.check(exa.exa_loglik_batched(ctx.handle, len(ns), ns, dl, dz, th, prec, out, st))
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


@pytest.fixture(scope="module")
def ctx():
    import paper_1908_06936_gb300 as exa

    c = exa.Context()
    yield c
    c.close()


@pytest.mark.parametrize("tile", [32, 64])
def test_batched_vs_oracle(ctx, tile):
    import paper_1908_06936_gb300 as exa

    sides = [5, 9, 12, 17, 20, 1, 3, 25, 8, 14]
    locs, zs = make_batch(sides, seed=10)
    thetas = synth.theta_perturbations((1.0, 0.1, 0.5), len(sides), seed=3)
    exa.exa_ctx_set_batched(ctx.handle, tile, 0, 0, 0)
    got, st = run(ctx, locs, zs, thetas)
    assert np.all(st == 0)
    for r in range(len(sides)):
        ref = oracle.loglik(locs[r], zs[r], thetas[r])["l"]
        assert abs(got[r] - ref) <= 1e-10 * abs(ref), (r, got[r], ref)
    exa.exa_ctx_set_batched(ctx.handle, 0, 0, 0, 0)


def test_batched_failures_are_per_replicate(ctx):
    sides = [6, 10, 7, 11]
    locs, zs = make_batch(sides, seed=20)
    locs[1][17, 0] = float("nan")
    thetas = np.tile([1.0, 0.1, 0.5], (4, 1))
    thetas[3, 1] = -0.2
    got, st = run(ctx, locs, zs, thetas)
    assert list(st) == [0, 2, 0, 1]
    assert math.isnan(got[1]) and math.isnan(got[3])
    for r in (0, 2):
        assert abs(got[r] - oracle.loglik(locs[r], zs[r], thetas[r])["l"]) <= 1e-10 * abs(got[r])


def test_batched_wait_times_out_and_context_survives(ctx):
    import paper_1908_06936_gb300 as exa

    sides = [8, 12, 16]
    locs, zs = make_batch(sides, seed=30)
    thetas = np.tile([1.0, 0.1, 0.5], (3, 1))
    exa.exa_ctx_set_batched(ctx.handle, 64, 0, 2_000_000, 1)  # ~1 ms waits, one task that never becomes ready
    try:
        got, st = run(ctx, locs, zs, thetas)
    finally:
        exa.exa_ctx_set_batched(ctx.handle, 0, 0, 0, 0)
    assert np.any(st == exa.EXA_ERR_TIMEOUT)
    assert all(math.isnan(got[r]) for r in range(3) if st[r] != 0)
    got2, st2 = run(ctx, locs, zs, thetas)
    assert np.all(st2 == 0)
    for r in range(3):
        assert abs(got2[r] - oracle.loglik(locs[r], zs[r], thetas[r])["l"]) <= 1e-10 * abs(got2[r])


def test_batched_graph_capture_replay_with_new_theta(ctx):
    import torch
    import paper_1908_06936_gb300 as exa

    sides = [7, 13, 10]
    locs, zs = make_batch(sides, seed=40)
    ns = [l.shape[0] for l in locs]
    dl = [to_dev(l) for l in locs]
    dz = [to_dev(z) for z in zs]
    th = to_dev(np.tile([1.0, 0.1, 0.5], 3))
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    st = torch.empty(3, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        exa.exa_ctx_set_stream(ctx.handle, s.cuda_stream)
        ctx.check(exa.exa_loglik_batched(ctx.handle, 3, ns, dl, dz, th, 0, out, st))  # allocates, outside capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ctx.check(exa.exa_loglik_batched(ctx.handle, 3, ns, dl, dz, th, 0, out, st))
    exa.exa_ctx_set_stream(ctx.handle, torch.cuda.current_stream().cuda_stream)
    for new in ([1.3, 0.08, 0.7], [0.6, 0.15, 1.2]):
        th.copy_(torch.tensor(new * 3, dtype=torch.float64))
        g.replay()
        torch.cuda.synchronize()
        res = out.cpu().numpy()
        for r in range(3):
            ref = oracle.loglik(locs[r], zs[r], new)["l"]
            assert abs(res[r] - ref) <= 1e-10 * abs(ref)


def test_batched_full_config_sigma2_scaling(ctx):
    # 256 replicates with n_i = m_i^2, m_i ~ U{20..80}: l(s) = a - (n/2) ln s - q/(2 s) holds
    # exactly for every replicate, so three sigma^2 values over-determine (a, q)
    sides = synth.replicate_sides(256, seed=5)
    locs = [synth.jittered_grid(int(m), 1000 + r) for r, m in enumerate(sides)]
    zs = [synth.normals(int(m) ** 2, 1000 + r) for r, m in enumerate(sides)]
    res = {}
    for s2 in (1.0, 2.0, 4.0):
        got, st = run(ctx, locs, zs, np.tile([s2, 0.1, 0.5], (256, 1)))
        assert np.all(st == 0)
        res[s2] = got
    n = np.array([l.shape[0] for l in locs], dtype=np.float64)
    # from s = 1 and s = 4: q = (8/3)(l4 - l1 + n ln 2); predict s = 2
    q = (8.0 / 3.0) * (res[4.0] - res[1.0] + n * math.log(2.0))
    a = res[1.0] + 0.5 * q
    pred2 = a - 0.5 * n * math.log(2.0) - q / 4.0
    assert np.all(np.abs(pred2 - res[2.0]) <= 1e-10 * np.abs(res[2.0]))
    # spot-check the smallest replicates against the oracle
    for r in np.argsort(n)[:3]:
        ref = oracle.loglik(locs[r], zs[r], (1.0, 0.1, 0.5))["l"]
        assert abs(res[1.0][r] - ref) <= 1e-10 * abs(ref)


# ---- mixed precision (FP32 off-diagonal tiles, FP64 diagonal tiles, FP64 refinement) ----
MIXED = 1  # EXA_MIXED_FP32
MIXED_TOL = 1e-6  # stated bound for a reduced-precision log-likelihood, |dl|/|l|


@pytest.mark.parametrize("tile", [32, 64])
def test_batched_mixed_vs_oracle(ctx, tile):
    import paper_1908_06936_gb300 as exa

    sides = [5, 9, 12, 17, 20, 1, 3, 25, 8, 14, 31]
    locs, zs = make_batch(sides, seed=50)
    thetas = synth.theta_perturbations((1.0, 0.1, 0.5), len(sides), seed=4)
    exa.exa_ctx_set_batched(ctx.handle, tile, 0, 0, 0)
    try:
        got, st = run(ctx, locs, zs, thetas, prec=MIXED)
    finally:
        exa.exa_ctx_set_batched(ctx.handle, 0, 0, 0, 0)
    assert np.all(st == 0), st
    for r in range(len(sides)):
        ref = oracle.loglik(locs[r], zs[r], thetas[r])["l"]
        assert abs(got[r] - ref) <= MIXED_TOL * abs(ref), (r, got[r], ref)


def test_batched_mixed_all_fp64_band_is_exact(ctx):
    # a band wider than every replicate keeps every tile in FP64: the refinement
    # then starts from an FP64 factor and the result matches the oracle to FP64 accuracy
    import paper_1908_06936_gb300 as exa

    sides = [6, 13, 22, 30]
    locs, zs = make_batch(sides, seed=60)
    thetas = synth.theta_perturbations((1.0, 0.1, 0.5), len(sides), seed=5)
    exa.exa_ctx_set_batched_mixed(ctx.handle, 1000, 0)
    try:
        got, st = run(ctx, locs, zs, thetas, prec=MIXED)
    finally:
        exa.exa_ctx_set_batched_mixed(ctx.handle, 0, 0)
    assert np.all(st == 0)
    for r in range(len(sides)):
        ref = oracle.loglik(locs[r], zs[r], thetas[r])["l"]
        assert abs(got[r] - ref) <= 1e-10 * abs(ref), (r, got[r], ref)


def test_batched_mixed_one_step_reports_unconverged(ctx):
    # one refinement step from an FP32 factor of a smooth field cannot reach the
    # 1e-8 residual: such replicates must say so (status 6, NaN), the rest be right
    import paper_1908_06936_gb300 as exa

    sides = [20, 24, 28]
    theta = (1.0, 0.3, 1.5)
    locs, zs = make_batch(sides, seed=70, theta0=theta)
    exa.exa_ctx_set_batched_mixed(ctx.handle, 0, 1)
    try:
        got, st = run(ctx, locs, zs, np.tile(theta, (3, 1)), prec=MIXED)
    finally:
        exa.exa_ctx_set_batched_mixed(ctx.handle, 0, 0)
    assert set(st.tolist()) <= {0, exa.EXA_ERR_IR_NOCONV, exa.EXA_ERR_NOT_SPD}
    for r in range(3):
        if st[r] == 0:
            ref = oracle.loglik(locs[r], zs[r], theta)["l"]
            assert abs(got[r] - ref) <= MIXED_TOL * abs(ref)
        else:
            assert math.isnan(got[r])


def test_batched_mixed_graph_replay(ctx):
    import torch
    import paper_1908_06936_gb300 as exa

    sides = [11, 19, 16]
    locs, zs = make_batch(sides, seed=80)
    ns = [l.shape[0] for l in locs]
    dl = [to_dev(l) for l in locs]
    dz = [to_dev(z) for z in zs]
    th = to_dev(np.tile([1.0, 0.1, 0.5], 3))
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    st = torch.empty(3, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        exa.exa_ctx_set_stream(ctx.handle, s.cuda_stream)
        ctx.check(exa.exa_loglik_batched(ctx.handle, 3, ns, dl, dz, th, MIXED, out, st))
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ctx.check(exa.exa_loglik_batched(ctx.handle, 3, ns, dl, dz, th, MIXED, out, st))
    exa.exa_ctx_set_stream(ctx.handle, torch.cuda.current_stream().cuda_stream)
    for new in ([1.3, 0.08, 0.7], [0.6, 0.15, 0.4]):
        th.copy_(torch.tensor(new * 3, dtype=torch.float64))
        g.replay()
        torch.cuda.synchronize()
        res, sts = out.cpu().numpy(), st.cpu().numpy()
        assert np.all(sts == 0)
        for r in range(3):
            ref = oracle.loglik(locs[r], zs[r], new)["l"]
            assert abs(res[r] - ref) <= MIXED_TOL * abs(ref)


def test_batched_mixed_full_config_vs_fp64(ctx):
    # 256 replicates, n_i = m_i^2 with m_i ~ U{20..80}, theta0 = (1, 0.1, 0.5), Z = L eps per replicate
    sides = synth.replicate_sides(256, seed=5)
    locs = [synth.jittered_grid(int(m), 1000 + r) for r, m in enumerate(sides)]
    zs = [synth.normals(int(m) ** 2, 1000 + r) for r, m in enumerate(sides)]
    th = np.tile([1.0, 0.1, 0.5], (256, 1))
    ref, st64 = run(ctx, locs, zs, th, prec=0)
    got, st = run(ctx, locs, zs, th, prec=MIXED)
    assert np.all(st64 == 0) and np.all(st == 0)
    rel = np.abs(got - ref) / np.abs(ref)
    assert rel.max() <= MIXED_TOL, (rel.max(), int(rel.argmax()))


def test_batched_rejects_bf16x3_and_unknown_precisions(ctx):
    import torch
    import paper_1908_06936_gb300 as exa

    locs, zs = make_batch([6], seed=90)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    th = to_dev(np.array([1.0, 0.1, 0.5]))
    for prec in (exa.EXA_MIXED_BF16X3, 7):
        rc = exa.exa_loglik_batched(ctx.handle, 1, [36], [to_dev(locs[0])], [to_dev(zs[0])], th, prec, out, st)
        assert rc == exa.EXA_ERR_ARG


# ---- tensor-core form (EXA_MIXED_TF32X3): grouped tcgen05 TF32x3 panel solves and updates ----
TC = 3  # EXA_MIXED_TF32X3


def test_batched_tc_vs_oracle(ctx):
    # uneven sizes, ragged tiles, one replicate of a single point, parameters perturbed per replicate
    sides = [5, 9, 12, 17, 20, 1, 3, 25, 8, 14, 31, 40]
    locs, zs = make_batch(sides, seed=51)
    thetas = synth.theta_perturbations((1.0, 0.1, 0.5), len(sides), seed=6)
    got, st = run(ctx, locs, zs, thetas, prec=TC)
    assert np.all(st == 0), st
    for r in range(len(sides)):
        ref = oracle.loglik(locs[r], zs[r], thetas[r])["l"]
        assert abs(got[r] - ref) <= MIXED_TOL * abs(ref), (r, got[r], ref)


def test_batched_tc_matches_the_persistent_forms(ctx):
    # the same batch through the FP64 persistent form, the FP32 persistent form and the tensor-core form
    sides = [20, 33, 47, 28, 60]
    locs, zs = make_batch(sides, seed=52)
    th = np.tile([1.0, 0.1, 0.5], (len(sides), 1))
    f64, s64 = run(ctx, locs, zs, th, prec=0)
    tc, stc = run(ctx, locs, zs, th, prec=TC)
    f32, s32 = run(ctx, locs, zs, th, prec=MIXED)
    tc2, stc2 = run(ctx, locs, zs, th, prec=TC)  # after the persistent form rebuilt its plan
    assert np.all(s64 == 0) and np.all(stc == 0) and np.all(s32 == 0) and np.all(stc2 == 0)
    assert np.array_equal(tc, tc2)  # bitwise repeatable
    assert np.all(np.abs(tc - f64) <= MIXED_TOL * np.abs(f64)), (tc, f64)


def test_batched_tc_not_spd_replicate_is_isolated(ctx):
    # a replicate with a non-finite location has a non-finite pivot: it reports EXA_ERR_NOT_SPD and
    # NaN, the others are unaffected
    import paper_1908_06936_gb300 as exa

    sides = [12, 15, 18]
    locs, zs = make_batch(sides, seed=53)
    locs[1] = locs[1].copy()
    locs[1][150, 0] = float("nan")
    th = np.tile([1.0, 0.1, 0.5], (3, 1))
    got, st = run(ctx, locs, zs, th, prec=TC)
    assert st[1] == exa.EXA_ERR_NOT_SPD and math.isnan(got[1])
    for r in (0, 2):
        assert st[r] == 0
        ref = oracle.loglik(locs[r], zs[r], (1.0, 0.1, 0.5))["l"]
        assert abs(got[r] - ref) <= MIXED_TOL * abs(ref)


def test_batched_tc_graph_replay(ctx):
    import torch
    import paper_1908_06936_gb300 as exa

    sides = [11, 19, 16, 30]
    locs, zs = make_batch(sides, seed=81)
    ns = [l.shape[0] for l in locs]
    dl = [to_dev(l) for l in locs]
    dz = [to_dev(z) for z in zs]
    th = to_dev(np.tile([1.0, 0.1, 0.5], 4))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    st = torch.empty(4, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        exa.exa_ctx_set_stream(ctx.handle, s.cuda_stream)
        ctx.check(exa.exa_loglik_batched(ctx.handle, 4, ns, dl, dz, th, TC, out, st))
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ctx.check(exa.exa_loglik_batched(ctx.handle, 4, ns, dl, dz, th, TC, out, st))
    exa.exa_ctx_set_stream(ctx.handle, torch.cuda.current_stream().cuda_stream)
    for new in ([1.3, 0.08, 0.7], [0.6, 0.15, 0.4]):
        th.copy_(torch.tensor(new * 4, dtype=torch.float64))
        g.replay()
        torch.cuda.synchronize()
        res, sts = out.cpu().numpy(), st.cpu().numpy()
        assert np.all(sts == 0)
        for r in range(4):
            ref = oracle.loglik(locs[r], zs[r], new)["l"]
            assert abs(res[r] - ref) <= MIXED_TOL * abs(ref)


def test_batched_tc_full_config_vs_fp64(ctx):
    # the 256-replicate configuration: every replicate within the mixed bound of the FP64 form
    sides = synth.replicate_sides(256, seed=5)
    locs = [synth.jittered_grid(int(m), 1000 + r) for r, m in enumerate(sides)]
    zs = [synth.normals(int(m) ** 2, 1000 + r) for r, m in enumerate(sides)]
    th = np.tile([1.0, 0.1, 0.5], (256, 1))
    ref, st64 = run(ctx, locs, zs, th, prec=0)
    got, st = run(ctx, locs, zs, th, prec=TC)
    assert np.all(st64 == 0) and np.all(st == 0)
    rel = np.abs(got - ref) / np.abs(ref)
    print("tensor-core batched: max |dl|/|l| = %.2e" % rel.max())
    assert rel.max() <= MIXED_TOL, (rel.max(), int(rel.argmax()))


def test_batched_autotune_picks_a_candidate_and_keeps_results(ctx, tmp_path):
    import torch
    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300 import tune

    sides = [8, 15, 21, 12]
    locs, zs = make_batch(sides, seed=95)
    ns = [l.shape[0] for l in locs]
    dl = [to_dev(l) for l in locs]
    dz = [to_dev(z) for z in zs]
    th = to_dev(np.tile([1.0, 0.1, 0.5], 4))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    st = torch.empty(4, dtype=torch.int32, device="cuda")
    try:
        r = tune.autotune_batched(ctx, ns, dl, dz, th, MIXED, out, st, cache_path=str(tmp_path / "t.json"))
        assert r["tile_nb"] in (32, 64) and r["ctas_per_sm"] >= 1 and r["ms"] > 0 and not r["cached"]
        r2 = tune.autotune_batched(ctx, ns, dl, dz, th, MIXED, out, st, cache_path=str(tmp_path / "t.json"))
        assert r2["cached"] and r2["tile_nb"] == r["tile_nb"]
        got, sts = run(ctx, locs, zs, np.tile([1.0, 0.1, 0.5], (4, 1)), prec=MIXED)
    finally:
        exa.exa_ctx_set_batched(ctx.handle, 0, 0, 0, 0)
    assert np.all(sts == 0)
    for r_ in range(4):
        ref = oracle.loglik(locs[r_], zs[r_], (1.0, 0.1, 0.5))["l"]
        assert abs(got[r_] - ref) <= MIXED_TOL * abs(ref)


def test_batched_autotune_tc_form_reports_its_single_configuration(ctx):
    # the tensor-core form has one configuration: autotune times it and leaves the persistent
    # forms' options alone
    import torch
    import paper_1908_06936_gb300 as exa

    sides = [8, 15, 21, 12]
    locs, zs = make_batch(sides, seed=96)
    ns = [l.shape[0] for l in locs]
    dl = [to_dev(l) for l in locs]
    dz = [to_dev(z) for z in zs]
    th = to_dev(np.tile([1.0, 0.1, 0.5], 4))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    st = torch.empty(4, dtype=torch.int32, device="cuda")
    ctx.check(exa.exa_ctx_set_batched(ctx.handle, 32, 1, 0, 0))
    try:
        rc, nb, cps, ms = exa.exa_batched_autotune(ctx.handle, 4, ns, dl, dz, th, TC, out, st)
        ctx.check(rc)
        assert nb == 128 and cps == 0 and ms > 0
        assert np.all(st.cpu().numpy() == 0)
        got = out.cpu().numpy()
        f32, s32 = run(ctx, locs, zs, np.tile([1.0, 0.1, 0.5], (4, 1)), prec=MIXED)  # still tile 32, 1 CTA/SM
        assert np.all(s32 == 0)
    finally:
        exa.exa_ctx_set_batched(ctx.handle, 0, 0, 0, 0)
    for r_ in range(4):
        ref = oracle.loglik(locs[r_], zs[r_], (1.0, 0.1, 0.5))["l"]
        assert abs(got[r_] - ref) <= MIXED_TOL * abs(ref)
        assert abs(f32[r_] - ref) <= MIXED_TOL * abs(ref)
