"""Host-side logic of the maximum-likelihood drivers: the ask/tell Nelder-Mead used to fit
many replicates in lockstep (no GPU; the objectives here are closed forms or the oracle)."""
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from paper_1908_06936_gb300.mle import NelderMead, fit_replicates_with


def run(nm, f):
    while not nm.done:
        nm.tell(f(nm.ask()))
    return nm.best()


def test_quadratic_minimum_found():
    a = np.array([0.3, -1.2, 2.0])
    w = np.array([1.0, 5.0, 0.5])
    nm = NelderMead([0.0, 0.0, 0.0], [0.5] * 3, [-10] * 3, [10] * 3, ftol=1e-12, xtol=1e-7, max_evals=5000)
    x, fx = run(nm, lambda x: float(np.sum(w * (x - a) ** 2)))
    assert np.max(np.abs(x - a)) < 1e-5 and fx < 1e-9


def test_rosenbrock_3d():
    def rb(x):
        return float(sum(100.0 * (x[i + 1] - x[i] ** 2) ** 2 + (1 - x[i]) ** 2 for i in range(2)))

    nm = NelderMead([-1.0, 1.5, 0.5], [0.5] * 3, [-5] * 3, [5] * 3, ftol=1e-14, xtol=1e-8, max_evals=20000)
    x, fx = run(nm, rb)
    assert np.max(np.abs(x - 1.0)) < 1e-4, x


def test_box_constrained_minimum_on_the_boundary():
    # unconstrained minimum at (2, 0, -3) lies outside [-1, 1]^3: the clipped search ends on the face
    a = np.array([2.0, 0.0, -3.0])
    nm = NelderMead([0.0, 0.5, 0.0], [0.3] * 3, [-1] * 3, [1] * 3, ftol=1e-12, xtol=1e-7, max_evals=5000)
    x, _ = run(nm, lambda x: float(np.sum((x - a) ** 2)))
    assert np.allclose(x, [1.0, 0.0, -1.0], atol=1e-5)
    assert np.all(x >= -1) and np.all(x <= 1)


def test_non_finite_region_is_avoided():
    # f = +inf wherever x0 > 0.5: the minimiser of (x - 1)^2 restricted to x0 <= 0.5
    def f(x):
        return math.inf if x[0] > 0.5 else float(np.sum((x - 1.0) ** 2))

    nm = NelderMead([0.0, 0.0, 0.0], [0.2] * 3, [-3] * 3, [3] * 3, ftol=1e-10, xtol=1e-6, max_evals=5000)
    x, fx = run(nm, f)
    assert math.isfinite(fx) and x[0] <= 0.5 and abs(x[0] - 0.5) < 1e-3 and np.allclose(x[1:], 1.0, atol=1e-3)


def test_evaluation_budget_is_respected():
    nm = NelderMead([0.0] * 3, [1.0] * 3, [-9] * 3, [9] * 3, ftol=0.0, xtol=0.0, max_evals=37)
    n = 0
    while not nm.done:
        nm.tell(float(np.sum(nm.ask() ** 2)) + 1.0)
        n += 1
    assert nm.evals == n and 37 <= n <= 37 + 3


def test_lockstep_fit_of_known_maxima():
    # replicate r's "log-likelihood" peaks at theta_r; the fitted theta must find each
    targets = np.array([[0.8, 0.05, 0.6], [1.5, 0.2, 1.1], [0.3, 0.02, 0.3]])

    def ll(r, th):
        return -float(np.sum((np.log(th) - np.log(targets[r])) ** 2))

    res = fit_replicates_with(ll, 3, x0=[1.0, 0.1, 0.5], ftol=1e-14, xtol=1e-8, max_evals=3000)
    assert np.allclose(res["theta"], targets, rtol=1e-5)


@pytest.mark.slow
def test_oracle_fit_is_a_local_maximum():
    m = 7
    locs = synth.jittered_grid(m, 3)
    z = oracle.simulate(locs, (1.0, 0.1, 0.5), synth.normals(m * m, 3))
    res = fit_replicates_with(lambda r, th: oracle.loglik(locs, z, th)["l"], 1, x0=[1.0, 0.1, 0.5],
                              ftol=1e-10, xtol=1e-6, max_evals=1500)
    th = res["theta"][0]
    l0 = oracle.loglik(locs, z, th)["l"]
    lo, hi = np.asarray(synth.THETA_LOWER), np.asarray(synth.THETA_UPPER)
    for k in range(3):
        for f in (0.99, 1.01):
            t = th.copy()
            t[k] = min(max(t[k] * f, lo[k]), hi[k])
            assert oracle.loglik(locs, z, t)["l"] <= l0 + 1e-9


class _OracleCtx:
    """Stands in for a library context in the single-field drivers: the same calls, answered by the oracle."""

    def loglik(self, locs, z, theta, prec=0):
        import paper_1908_06936_gb300 as exa

        r = oracle.loglik(locs, z, theta)
        if r["info"] != 0:
            raise exa.ExaError(exa.EXA_ERR_NOT_SPD, "not SPD")
        return r["l"]

    def loglik_grad(self, locs, z, theta, prec=0):
        r = oracle.loglik_grad(locs, z, theta)
        return r["l"], np.asarray(r["grad"])


@pytest.mark.parametrize("driver", ["derivative_free", "gradient"])
def test_history_file_records_every_evaluation_and_resumes_from_its_best(tmp_path, driver):
    from paper_1908_06936_gb300 import mle

    locs = synth.jittered_grid(8, seed=3)
    z = oracle.simulate(locs, (1.0, 0.1, 0.5), synth.normals(64, 3))
    path = str(tmp_path / "fit.jsonl")
    if driver == "derivative_free":
        fit = lambda: mle.fit_derivative_free(locs, z, maxfev=25, ctx=_OracleCtx(), history_path=path)
    else:
        fit = lambda: mle.fit_gradient(locs, z, maxiter=4, ctx=_OracleCtx(), history_path=path)
    a = fit()
    assert a["resumed_from"] is None
    rows = mle.load_history(path)
    assert len(rows) == a["evals"] == len(a["history"]) > 0
    for (th_f, l_f), (th_m, l_m) in zip(rows, a["history"]):
        assert np.allclose(th_f, th_m, rtol=0, atol=0) and (l_f == l_m or (math.isinf(l_f) and math.isinf(l_m)))
    best = mle.best_in_history(path)
    assert best[1] == max(l for _, l in rows if math.isfinite(l))
    # a second run on the same file starts from that best theta and appends its own evaluations
    b = fit()
    assert b["resumed_from"] == best[0]
    assert np.allclose(b["history"][0][0], best[0], rtol=1e-12, atol=0)
    assert len(mle.load_history(path)) == a["evals"] + b["evals"]
    assert b["loglik"] >= best[1] - 1e-9


def test_history_keeps_non_finite_evaluations(tmp_path):
    from paper_1908_06936_gb300 import mle

    path = str(tmp_path / "h.jsonl")
    h = mle.EvalHistory(path)
    h.append(([1.0, 0.1, 0.5], -12.5))
    h.append(([2.0, 0.3, 1.0], -math.inf))
    assert mle.load_history(path) == [([1.0, 0.1, 0.5], -12.5), ([2.0, 0.3, 1.0], -math.inf)]
    assert mle.best_in_history(path) == ([1.0, 0.1, 0.5], -12.5)
    assert mle.best_in_history(str(tmp_path / "absent.jsonl")) is None
