"""Degenerate and invalid observations through the C ABI.

z = 0 is the degenerate case of Eq. 2: the quadratic form vanishes and l is the normalising term
-n/2 log 2 pi - 1/2 log|Sigma| alone, so every path must return q = 0 exactly (the mixed path has nothing to
refine).  A z holding a non-finite entry is an argument error (EXA_ERR_ARG, l = NaN), not a NaN result with
EXA_OK, and the context stays usable after it.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from gpu_util import to_dev, workload

pytestmark = pytest.mark.gpu

THETA = (1.0, 0.1, 0.5)


@pytest.mark.parametrize("prec_name,tol", [("EXA_FP64", 1e-10), ("EXA_MIXED_TF32X3", 1e-6)])
def test_zero_observations(prec_name, tol):
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(40, seed=3)
    z = np.zeros(1600)
    ref = oracle.loglik(locs, z, THETA)
    assert ref["quad"] == 0.0
    with exa.Context() as c:
        got = c.loglik_ex(to_dev(locs), to_dev(z), THETA, getattr(exa, prec_name))
    assert got["quad"] == 0.0 and got["quad_err"] == 0.0
    assert abs(got["logdet"] - ref["logdet"]) <= tol * abs(ref["logdet"])
    assert abs(got["loglik"] - ref["l"]) <= tol * abs(ref["l"])


@pytest.mark.parametrize("prec_name", ["EXA_FP64", "EXA_MIXED_TF32X3"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_observation_is_an_argument_error(prec_name, bad):
    import paper_1908_06936_gb300 as exa

    locs, z = workload(20, seed=4)
    z = z.copy()
    z[123] = bad
    prec = getattr(exa, prec_name)
    with exa.Context() as c:
        with pytest.raises(exa.ExaError) as ei:
            c.loglik(to_dev(locs), to_dev(z), THETA, prec)
        assert ei.value.status == exa.EXA_ERR_ARG
        # the same context evaluates the corrected field
        z[123] = 0.5
        ref = oracle.loglik(locs, z, THETA)["l"]
        assert abs(c.loglik(to_dev(locs), to_dev(z), THETA, prec) - ref) <= 1e-6 * abs(ref)


def test_non_finite_observation_allocation_free_entry():
    import torch
    import paper_1908_06936_gb300 as exa

    locs, z = workload(12, seed=5)
    z = z.copy()
    z[7] = float("nan")
    out = ctypes.c_double()
    st = exa.exa_loglik_noalloc(torch.cuda.current_stream().cuda_stream, to_dev(locs), to_dev(z), THETA, 144, out)
    assert st == exa.EXA_ERR_ARG and math.isnan(out.value)
