"""Maximum-likelihood drivers (host control only; every evaluation runs in the library).

The paper maximises l(theta) with NLopt's BOBYQA, a bounded derivative-free
trust-region method, starting from the lower bounds (Section II-B, Section III
Example 2).  Two drivers are offered over the same bounds:

* ``fit_derivative_free``: scipy's bounded Nelder-Mead or Powell on -l(theta);
* ``fit_gradient``: scipy's L-BFGS-B on -l(theta) with the library's analytic
  gradient (exa_loglik_grad).

Evaluations that are not SPD return l = -inf (the optimiser steps away).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import EXA_FP64, Context, ExaError
from .synth import THETA_LOWER, THETA_UPPER


def _objective(ctx, locs, z, prec, history):
    def f(th):
        th = np.clip(np.asarray(th, dtype=np.float64), THETA_LOWER, THETA_UPPER)
        try:
            l = ctx.loglik(locs, z, th.tolist(), prec)
        except ExaError as e:
            if e.status in (2, 6):  # not SPD / refinement stalled: outside the usable region
                l = -math.inf
            else:
                raise
        history.append((th.tolist(), l))
        return -l if math.isfinite(l) else 1e300
    return f


def fit_derivative_free(locs, z, x0=None, prec=EXA_FP64, method="Nelder-Mead", maxfev=100, ftol_abs=1e-4,
                        ctx: Context | None = None) -> dict:
    from scipy.optimize import minimize

    c = ctx or Context()
    hist: list = []
    x0 = np.asarray(THETA_LOWER if x0 is None else x0, dtype=np.float64)
    t0 = time.perf_counter()
    opts = {"maxfev": maxfev, "fatol": ftol_abs, "xatol": 1e-6} if method == "Nelder-Mead" else \
        {"maxfev": maxfev, "ftol": 1e-10}
    r = minimize(_objective(c, locs, z, prec, hist), x0, method=method,
                 bounds=list(zip(THETA_LOWER, THETA_UPPER)), options=opts)
    dt = time.perf_counter() - t0
    if ctx is None:
        c.close()
    return {"theta": np.clip(r.x, THETA_LOWER, THETA_UPPER).tolist(), "loglik": -r.fun, "evals": len(hist),
            "seconds": dt, "time_per_eval": dt / max(1, len(hist)), "history": hist, "method": method}


def fit_gradient(locs, z, x0=None, maxiter=100, ctx: Context | None = None) -> dict:
    from scipy.optimize import minimize

    c = ctx or Context()
    hist: list = []

    def fg(th):
        th = np.clip(np.asarray(th, dtype=np.float64), THETA_LOWER, THETA_UPPER)
        try:
            l, g = c.loglik_grad(locs, z, th.tolist())
        except ExaError as e:
            if e.status == 2:
                hist.append((th.tolist(), -math.inf))
                return 1e300, np.zeros(3)
            raise
        hist.append((th.tolist(), l))
        return -l, -np.asarray(g)

    x0 = np.asarray(THETA_LOWER if x0 is None else x0, dtype=np.float64)
    t0 = time.perf_counter()
    r = minimize(fg, x0, jac=True, method="L-BFGS-B", bounds=list(zip(THETA_LOWER, THETA_UPPER)),
                 options={"maxiter": maxiter})
    dt = time.perf_counter() - t0
    if ctx is None:
        c.close()
    return {"theta": r.x.tolist(), "loglik": -r.fun, "evals": len(hist), "seconds": dt,
            "time_per_eval": dt / max(1, len(hist)), "history": hist, "method": "L-BFGS-B+analytic gradient"}
