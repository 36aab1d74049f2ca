"""Fisher information (exact_fisher) through the C ABI against the oracle, plus the sigma^2
closed form I_11 = n / (2 sigma^4) at a size beyond the oracle's reach."""
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


@pytest.mark.parametrize("m,theta", [(7, (1.0, 0.1, 0.5)), (19, (1.5, 0.2, 1.5)), (26, (0.7, 0.05, 0.9))])
def test_fisher_vs_oracle(ctx, m, theta):
    locs = synth.jittered_grid(m, m)
    ref = oracle.fisher(locs, theta)
    got = ctx.fisher(to_dev(locs), theta)
    assert np.allclose(got, got.T, rtol=0, atol=0)
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(got - ref) <= 1e-9 * scale), np.max(np.abs(got - ref) / scale)


def test_fisher_sigma2_closed_form_large(ctx):
    theta = (2.5, 0.1, 0.8)
    locs = synth.jittered_grid(60, 3)
    got = ctx.fisher(to_dev(locs), theta)
    assert abs(got[0, 0] - 3600 / (2 * theta[0] ** 2)) <= 1e-9 * got[0, 0]
    assert np.all(np.linalg.eigvalsh(got) > 0)


def test_fisher_arguments(ctx):
    import paper_1908_06936_gb300 as exa

    locs = synth.jittered_grid(4, 1)
    with pytest.raises(exa.ExaError):
        ctx.fisher(to_dev(locs), (1.0, 0.0, 0.5))
    locs[2, 1] = float("nan")
    with pytest.raises(exa.ExaError):
        ctx.fisher(to_dev(locs), (1.0, 0.1, 0.5))
