"""Maximum-likelihood drivers (host control only; every evaluation runs in the library).

The paper maximises l(theta) with NLopt's BOBYQA, a bounded derivative-free
trust-region method, starting from the lower bounds (Section II-B, Section III
Example 2).  Two drivers are offered over the same bounds:

* ``fit_derivative_free``: scipy's bounded Nelder-Mead or Powell on -l(theta);
* ``fit_gradient``: scipy's L-BFGS-B on -l(theta) with the library's analytic
  gradient (exa_loglik_grad).

Evaluations that are not SPD return l = -inf (the optimiser steps away).

With ``history_path`` every evaluation is also appended to that file as one JSON
line, so a fit that was interrupted restarts from the best theta recorded there.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import EXA_FP64, Context, ExaError
from .synth import THETA_LOWER, THETA_UPPER


class EvalHistory:
    """The (theta, l) of every evaluation of one fit, in order.  With a path, each evaluation is also
    appended to that file as a JSON line {"theta": [...], "loglik": l} (null where l is not finite) and
    flushed at once, so the record survives an interrupted run."""

    def __init__(self, path: str | None = None):
        self.rows: list = []
        self.path = path

    def append(self, row) -> None:
        theta, l = row
        self.rows.append((list(theta), l))
        if self.path:
            with open(self.path, "a") as f:
                f.write(json.dumps({"theta": [float(v) for v in theta],
                                    "loglik": float(l) if math.isfinite(l) else None}) + "\n")

    def __len__(self) -> int:
        return len(self.rows)


def load_history(path: str) -> list:
    """The (theta, l) rows of a history file, in order (l = -inf where none was recorded)."""
    rows = []
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                if line.strip():
                    d = json.loads(line)
                    rows.append((d["theta"], -math.inf if d["loglik"] is None else float(d["loglik"])))
    return rows


def best_in_history(path: str):
    """(theta, l) with the largest finite l in a history file, or None."""
    rows = [r for r in load_history(path) if math.isfinite(r[1])]
    return max(rows, key=lambda r: r[1]) if rows else None


def _start(x0, history_path):
    """The starting theta: x0 if given, else the best theta of an existing history, else the lower bounds."""
    if x0 is not None:
        return np.asarray(x0, dtype=np.float64), None
    best = best_in_history(history_path) if history_path else None
    if best is not None:
        return np.asarray(best[0], dtype=np.float64), best[0]
    return np.asarray(THETA_LOWER, dtype=np.float64), None


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
                        ctx: Context | None = None, history_path: str | None = None) -> dict:
    from scipy.optimize import minimize

    c = ctx or Context()
    hist = EvalHistory(history_path)
    x0, resumed = _start(x0, history_path)
    t0 = time.perf_counter()
    opts = {"maxfev": maxfev, "fatol": ftol_abs, "xatol": 1e-6} if method == "Nelder-Mead" else \
        {"maxfev": maxfev, "ftol": 1e-10}
    r = minimize(_objective(c, locs, z, prec, hist), x0, method=method,
                 bounds=list(zip(THETA_LOWER, THETA_UPPER)), options=opts)
    dt = time.perf_counter() - t0
    if ctx is None:
        c.close()
    return {"theta": np.clip(r.x, THETA_LOWER, THETA_UPPER).tolist(), "loglik": -r.fun, "evals": len(hist),
            "seconds": dt, "time_per_eval": dt / max(1, len(hist)), "history": hist.rows, "method": method,
            "resumed_from": resumed}


def fit_gradient(locs, z, x0=None, maxiter=100, ctx: Context | None = None, prec=EXA_FP64,
                 history_path: str | None = None) -> dict:
    """L-BFGS-B with the library's analytic gradient, in u = log(theta) (the three parameters span
    orders of magnitude between the bounds; the chain rule gives dl/du = theta * dl/dtheta) on the
    objective -l / n.  Evaluations that are not SPD (or whose refinement stalls) return a large
    value and a zero gradient, so the line search steps back."""
    from scipy.optimize import minimize

    c = ctx or Context()
    hist = EvalHistory(history_path)
    n = float(locs.shape[0])
    lo, hi = np.log(THETA_LOWER), np.log(THETA_UPPER)

    def fg(u):
        th = np.exp(np.clip(np.asarray(u, dtype=np.float64), lo, hi))
        try:
            l, g = c.loglik_grad(locs, z, th.tolist(), prec)
        except ExaError as e:
            if e.status in (2, 6):  # not SPD / refinement stalled: outside the usable region
                hist.append((th.tolist(), -math.inf))
                return 1e10, np.zeros(3)
            raise
        hist.append((th.tolist(), l))
        return -l / n, -(th * np.asarray(g)) / n

    x0, resumed = _start(x0, history_path)
    t0 = time.perf_counter()
    r = minimize(fg, np.log(x0), jac=True, method="L-BFGS-B", bounds=list(zip(lo, hi)),
                 options={"maxiter": maxiter})
    dt = time.perf_counter() - t0
    if ctx is None:
        c.close()
    th = np.exp(np.clip(r.x, lo, hi))
    return {"theta": th.tolist(), "loglik": -r.fun * n, "evals": len(hist), "seconds": dt,
            "time_per_eval": dt / max(1, len(hist)), "history": hist.rows,
            "method": "L-BFGS-B in log(theta) + analytic gradient", "message": str(r.message),
            "resumed_from": resumed}


# ---------------------------------------------------------------------------
# Many replicates at once (Section III, Example 2 fits every replicate field
# separately).  Each replicate runs its own bounded Nelder-Mead in log(theta);
# the minimisers advance in lockstep, so one batched evaluation (one CUDA-graph
# replay of exa_loglik_batched) serves one step of all of them.
# ---------------------------------------------------------------------------
class NelderMead:
    """One Nelder-Mead minimisation driven by ask() / tell(f), with the standard
    coefficients (reflection 1, expansion 2, contraction 1/2, shrink 1/2) and the
    acceptance rules of Lagarias, Reeds, Wright and Wright (1998).  Points are
    clipped into the box [lo, hi]; a non-finite f counts as +inf.  Stops when the
    simplex's f values span at most ftol and its vertices lie within xtol of the
    best one (max norm), or after max_evals evaluations."""

    def __init__(self, x0, step, lo, hi, ftol=1e-5, xtol=1e-4, max_evals=400):
        self.lo, self.hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
        x0 = self._clip(np.asarray(x0, dtype=np.float64))
        n = x0.size
        self.pts = [x0]
        for i in range(n):
            v = x0.copy()
            v[i] += step[i]
            if v[i] > self.hi[i]:  # no room above: step down instead
                v[i] = x0[i] - step[i]
            self.pts.append(self._clip(v))
        self.f = [math.inf] * (n + 1)
        self.ftol, self.xtol, self.max_evals = ftol, xtol, max_evals
        self.evals, self.done = 0, False
        self.phase, self.idx = "init", 0
        self._pending = self.pts[0]

    def _clip(self, x):
        return np.minimum(np.maximum(x, self.lo), self.hi)

    def best(self):
        i = int(np.argmin(self.f))
        return self.pts[i].copy(), self.f[i]

    def ask(self):
        return (self.best()[0] if self.done else self._pending).copy()

    def _start_iteration(self):
        order = np.argsort(self.f, kind="stable")
        self.pts = [self.pts[i] for i in order]
        self.f = [self.f[i] for i in order]
        spread_f = self.f[-1] - self.f[0]
        spread_x = max(float(np.max(np.abs(p - self.pts[0]))) for p in self.pts[1:])
        if (math.isfinite(spread_f) and spread_f <= self.ftol and spread_x <= self.xtol) or \
                self.evals >= self.max_evals:
            self.done = True
            return
        self.c = np.mean(self.pts[:-1], axis=0)
        self.xr = self._clip(self.c + (self.c - self.pts[-1]))
        self.phase, self._pending = "reflect", self.xr

    def _replace_worst(self, x, fx):
        self.pts[-1], self.f[-1] = x, fx
        self._start_iteration()

    def _shrink(self):
        x0 = self.pts[0]
        self.pts = [x0] + [self._clip(x0 + 0.5 * (p - x0)) for p in self.pts[1:]]
        self.phase, self.idx = "shrink", 1
        self._pending = self.pts[1]

    def tell(self, fx):
        if self.done:
            return
        fx = float(fx) if math.isfinite(fx) else math.inf
        self.evals += 1
        ph = self.phase
        if ph == "init":
            self.f[self.idx] = fx
            self.idx += 1
            if self.idx < len(self.pts):
                self._pending = self.pts[self.idx]
            else:
                self._start_iteration()
        elif ph == "reflect":
            self.fr = fx
            f1, fn, fw = self.f[0], self.f[-2], self.f[-1]
            if f1 <= fx < fn:
                self._replace_worst(self.xr, fx)
            elif fx < f1:
                self.xe = self._clip(self.c + 2.0 * (self.xr - self.c))
                self.phase, self._pending = "expand", self.xe
            elif fx < fw:
                self.xc = self._clip(self.c + 0.5 * (self.xr - self.c))
                self.phase, self._pending = "outside", self.xc
            else:
                self.xc = self._clip(self.c + 0.5 * (self.pts[-1] - self.c))
                self.phase, self._pending = "inside", self.xc
        elif ph == "expand":
            if fx < self.fr:
                self._replace_worst(self.xe, fx)
            else:
                self._replace_worst(self.xr, self.fr)
        elif ph == "outside":
            if fx <= self.fr:
                self._replace_worst(self.xc, fx)
            else:
                self._shrink()
        elif ph == "inside":
            if fx < self.f[-1]:
                self._replace_worst(self.xc, fx)
            else:
                self._shrink()
        elif ph == "shrink":
            self.f[self.idx] = fx
            self.idx += 1
            if self.idx < len(self.pts):
                self._pending = self.pts[self.idx]
            else:
                self._start_iteration()


def _log_box():
    return np.log(np.asarray(THETA_LOWER)), np.log(np.asarray(THETA_UPPER))


def fit_replicates(ns, locs_list, z_list, prec, x0=None, step=0.5, ftol=1e-5, xtol=1e-4, max_evals=400,
                   ctx: Context | None = None) -> dict:
    """Fit theta for every replicate at once: per step, one batched evaluation of all
    replicates (each at its own minimiser's point), replayed from a CUDA graph with the
    device theta array refilled in place.  x0 defaults to the lower bounds (as in the
    paper's examples); the search runs in log(theta) with initial steps `step`."""
    import torch

    from . import exa_ctx_set_stream, exa_loglik_batched

    nrep = len(ns)
    c = ctx or Context()
    lo, hi = _log_box()
    start = np.log(np.asarray(THETA_LOWER if x0 is None else x0, dtype=np.float64))
    nms = [NelderMead(start, [step] * 3, lo, hi, ftol=ftol, xtol=xtol, max_evals=max_evals) for _ in range(nrep)]
    th_host = torch.empty(3 * nrep, dtype=torch.float64).pin_memory()
    th = torch.empty(3 * nrep, dtype=torch.float64, device="cuda")
    out = torch.empty(nrep, dtype=torch.float64, device="cuda")
    st = torch.empty(nrep, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    steps = 0
    t0 = time.perf_counter()
    try:
        with torch.cuda.stream(s):
            exa_ctx_set_stream(c.handle, s.cuda_stream)
            th_host.copy_(torch.as_tensor(np.exp(np.concatenate([nm.ask() for nm in nms]))))
            th.copy_(th_host, non_blocking=True)
            c.check(exa_loglik_batched(c.handle, nrep, ns, locs_list, z_list, th, prec, out, st))  # allocates
            s.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                c.check(exa_loglik_batched(c.handle, nrep, ns, locs_list, z_list, th, prec, out, st))
            while not all(nm.done for nm in nms):
                pts = [nm.ask() for nm in nms]
                th_host.copy_(torch.as_tensor(np.exp(np.concatenate(pts))))
                th.copy_(th_host, non_blocking=True)
                g.replay()
                l = out.cpu().numpy()
                ok = st.cpu().numpy() == 0
                for r, nm in enumerate(nms):
                    nm.tell(-l[r] if ok[r] else math.inf)
                steps += 1
            s.synchronize()
    finally:
        exa_ctx_set_stream(c.handle, torch.cuda.current_stream().cuda_stream)
        if ctx is None:
            c.close()
    dt = time.perf_counter() - t0
    best = [nm.best() for nm in nms]
    return {"theta": np.exp(np.array([b[0] for b in best])), "loglik": np.array([-b[1] for b in best]),
            "evals": np.array([nm.evals for nm in nms]), "steps": steps, "seconds": dt,
            "replicate_evals_per_s": steps * nrep / dt}


def fit_replicates_with(loglik_fn, nrep, x0=None, step=0.5, ftol=1e-5, xtol=1e-4, max_evals=400) -> dict:
    """The same lockstep minimisers over any evaluator loglik_fn(r, theta) -> l (or
    -inf); used to run the identical search against a reference evaluator."""
    lo, hi = _log_box()
    start = np.log(np.asarray(THETA_LOWER if x0 is None else x0, dtype=np.float64))
    nms = [NelderMead(start, [step] * 3, lo, hi, ftol=ftol, xtol=xtol, max_evals=max_evals) for _ in range(nrep)]
    steps = 0
    while not all(nm.done for nm in nms):
        for r, nm in enumerate(nms):
            if nm.done:
                continue
            l = loglik_fn(r, np.exp(nm.ask()))
            nm.tell(-l if math.isfinite(l) else math.inf)
        steps += 1
    best = [nm.best() for nm in nms]
    return {"theta": np.exp(np.array([b[0] for b in best])), "loglik": np.array([-b[1] for b in best]),
            "evals": np.array([nm.evals for nm in nms]), "steps": steps}
