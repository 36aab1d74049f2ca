"""Writes the stored expected values under tests/golden/ from the FP64 oracle alone.

Run from the repository root:  python tests/golden/make_golden.py

Inputs come from the seeded generators of paper_1908_06936_gb300.synth (no method arithmetic there); every
number written is computed by oracle/ and nothing else.  The workload is the small-problem configuration of
Section III, Example 2: n = 1,600 locations (a 40 x 40 grid on [0,1]^2, jittered), sigma^2 = 1, and the field
Z = L eps drawn at theta0 = (1, 0.1, 0.5).  The values are the Eq. 2 log-likelihood with its two parts
(log det Sigma and Z^T Sigma^-1 Z) at theta0 and ten perturbations, and the gradient of Eq. 2 with respect to
(sigma^2, beta, nu) at theta0.

If the oracle's arithmetic is ever changed on purpose, rerun this script and name in the commit message the
passage of the paper (or the reading of it) that justifies the change.
"""
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(_HERE)))

import oracle  # noqa: E402
from paper_1908_06936_gb300 import synth  # noqa: E402

M, SEED = 40, 0
THETA0 = (1.0, 0.1, 0.5)
N_PERTURB = 10
OUT = os.path.join(_HERE, "config1_loglik_n1600.txt")


def thetas():
    return [THETA0] + [tuple(float(v) for v in t) for t in synth.theta_perturbations(THETA0, N_PERTURB, seed=SEED)]


def workload():
    locs = synth.jittered_grid(M, SEED)
    eps = synth.normals(M * M, SEED)
    return locs, oracle.simulate(locs, THETA0, eps)


def main():
    locs, Z = workload()
    lines = [
        "# Eq. 2 log-likelihood (zero mean) on the Section III, Example 2 small-problem setting:",
        "# n = 1600, 40 x 40 jittered grid on [0,1]^2 (synth.jittered_grid(40, 0)),",
        "# Z = L eps at theta0 = (1, 0.1, 0.5) with eps = synth.normals(1600, 0);",
        "# thetas = theta0 then synth.theta_perturbations(theta0, 10, seed=0).",
        "# Written by tests/golden/make_golden.py from the FP64 oracle only.",
        "# columns: kind sigma2 beta nu value(s)",
    ]
    for th in thetas():
        r = oracle.loglik(locs, Z, th)
        assert r["info"] == 0, th
        lines.append("loglik %s %s %s" % (" ".join(repr(float(v)) for v in th),
                                         " ".join(repr(float(r[k])) for k in ("l", "logdet", "quad")), ""))
    g = oracle.loglik_grad(locs, Z, THETA0)
    assert g["info"] == 0
    lines.append("grad %s %s" % (" ".join(repr(float(v)) for v in THETA0), " ".join(repr(float(v)) for v in g["grad"])))
    with open(OUT, "w") as f:
        f.write("\n".join(s.rstrip() for s in lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
