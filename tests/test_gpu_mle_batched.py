"""Lockstep maximum-likelihood fits of many replicates through the batched form (one
CUDA-graph replay per optimiser step) against the same search driven by the oracle."""
import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

THETA_TRUE = (1.0, 0.1, 0.5)
X0 = (0.5, 0.05, 0.8)


def replicates(sides, seed):
    locs, zs = [], []
    for r, m in enumerate(sides):
        l = synth.jittered_grid(int(m), seed + r)
        locs.append(l)
        zs.append(oracle.simulate(l, THETA_TRUE, synth.normals(int(m) ** 2, seed + r)))
    return locs, zs


def test_batched_fit_follows_the_oracle_search():
    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300.mle import fit_replicates, fit_replicates_with

    sides = [6, 9, 12, 15]
    locs, zs = replicates(sides, 300)
    ns = [l.shape[0] for l in locs]
    kw = dict(x0=X0, ftol=1e-7, xtol=1e-5, max_evals=200)
    gpu = fit_replicates(ns, [to_dev(l) for l in locs], [to_dev(z) for z in zs], exa.EXA_FP64, **kw)
    ref = fit_replicates_with(lambda r, th: oracle.loglik(locs[r], zs[r], th)["l"], len(sides), **kw)
    # FP64 likelihoods agree to ~1e-12, so both searches take the same path
    assert np.allclose(gpu["theta"], ref["theta"], rtol=1e-6), (gpu["theta"], ref["theta"])
    assert np.allclose(gpu["loglik"], ref["loglik"], rtol=1e-10)
    assert gpu["steps"] >= int(np.max(gpu["evals"]))


def test_batched_fit_mixed_precision_lands_on_the_same_maximum():
    import paper_1908_06936_gb300 as exa
    from paper_1908_06936_gb300.mle import fit_replicates

    sides = [10, 14, 18]
    locs, zs = replicates(sides, 400)
    ns = [l.shape[0] for l in locs]
    dl, dz = [to_dev(l) for l in locs], [to_dev(z) for z in zs]
    kw = dict(x0=X0, ftol=1e-7, xtol=1e-5, max_evals=300)
    f64 = fit_replicates(ns, dl, dz, exa.EXA_FP64, **kw)
    mix = fit_replicates(ns, dl, dz, exa.EXA_MIXED_FP32, **kw)
    assert np.allclose(mix["loglik"], f64["loglik"], rtol=1e-7)
    assert np.allclose(mix["theta"], f64["theta"], rtol=2e-2)
