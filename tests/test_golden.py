"""The oracle against the stored values in tests/golden/ (written by tests/golden/make_golden.py from the
oracle alone), and the stored values against relations Eq. 2 fixes by itself.

A difference from the stored file means the oracle's arithmetic changed: regenerate the file only when that
change is intended, naming the passage of the paper that justifies it.
"""
import math
import os
import sys

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_golden  # noqa: E402

N = make_golden.M * make_golden.M


def _rows():
    rows = []
    with open(os.path.join(GOLDEN, "config1_loglik_n1600.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kind, *vals = line.split()
            rows.append((kind, tuple(float(v) for v in vals[:3]), np.array([float(v) for v in vals[3:]])))
    return rows


ROWS = _rows()
LOGLIK = [(th, v) for k, th, v in ROWS if k == "loglik"]
GRAD = [(th, v) for k, th, v in ROWS if k == "grad"]


@pytest.fixture(scope="module")
def data():
    return make_golden.workload()


def test_file_covers_theta0_and_perturbations():
    assert [th for th, _ in LOGLIK] == make_golden.thetas()
    assert len(GRAD) == 1 and GRAD[0][0] == make_golden.THETA0


@pytest.mark.parametrize("th,v", LOGLIK)
def test_stored_values_obey_eq2(th, v):
    """l = -(log det Sigma + Z^T Sigma^-1 Z + n log 2 pi) / 2, term by term as Eq. 2 writes it."""
    l, logdet, quad = v
    assert quad > 0
    assert abs(l + 0.5 * (logdet + quad + N * math.log(2.0 * math.pi))) <= 1e-12 * abs(l)


def test_stored_sigma2_gradient_closed_form():
    """Sigma is linear in sigma^2, so dl/dsigma^2 = (Z^T Sigma^-1 Z - n) / (2 sigma^2)."""
    th, g = GRAD[0]
    quad = dict(LOGLIK)[th][2]
    assert abs(g[0] - (quad - N) / (2.0 * th[0])) <= 1e-10 * abs(g[0])


@pytest.mark.parametrize("th,v", LOGLIK)
def test_oracle_matches_stored_loglik(data, th, v):
    locs, Z = data
    r = oracle.loglik(locs, Z, th)
    assert r["info"] == 0
    got = np.array([r["l"], r["logdet"], r["quad"]])
    assert np.all(np.abs(got - v) <= 1e-12 * np.abs(v)), (th, got, v)


def test_oracle_matches_stored_gradient(data):
    locs, Z = data
    th, g = GRAD[0]
    r = oracle.loglik_grad(locs, Z, th)
    assert r["info"] == 0
    assert np.all(np.abs(r["grad"] - g) <= 1e-10 * np.max(np.abs(g))), (r["grad"], g)


def test_oracle_is_bitwise_independent_of_the_thread_count(data):
    """The oracle's OpenMP loops split only independent rows and columns, each computed in the serial order,
    so one thread and many give the same bits (the stored values do not depend on the machine's core count)."""
    import subprocess

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r); import make_golden, oracle; "
            "locs, Z = make_golden.workload(); r = oracle.loglik_grad(locs, Z, make_golden.THETA0); "
            "print(oracle.max_threads(), *[float(v).hex() for v in (r['l'], r['logdet'], r['quad'], *r['grad'])])"
            % (root, GOLDEN))
    one = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, OMP_NUM_THREADS="1"),
                         capture_output=True, text=True, timeout=600, check=True).stdout.split()
    assert one[0] == "1"
    locs, Z = data
    r = oracle.loglik_grad(locs, Z, make_golden.THETA0)
    many = [float(v).hex() for v in (r["l"], r["logdet"], r["quad"], *r["grad"])]
    assert one[1:] == many, (one, many, oracle.max_threads())
