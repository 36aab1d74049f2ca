"""Planted mistakes in the oracle must be caught by its pins.

Each case copies oracle/ into a temporary directory, plants one plausible mistake in oracle.c (a dropped term,
a wrong sign, order or index, a transposed operand), compiles it, and runs the pin tests that cover that
function against the mutated copy in a fresh interpreter.  The pins compare the oracle with things other than
itself (closed forms, DLMF identities, mpmath/scipy/LAPACK, brute force, invariants of Eq. 2), so every
mistake must turn at least one of them red.  The unmutated copy, through the same machinery, must stay green.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")
MODEL = os.path.join(ROOT, "tests", "test_oracle_model.py")
PREDICT = os.path.join(ROOT, "tests", "test_oracle_predict.py")
FISHER = os.path.join(ROOT, "tests", "test_oracle_fisher.py")

# (name, pin files, text in oracle.c, replacement, occurrences replaced)
MUTANTS = [
    ("Eq. 2: n/2 log 2pi dropped",
     [PINS], "ORACLE_LN_2PI = 1.8378770664093454835606594728112;", "ORACLE_LN_2PI = 0.0;", 1),
    ("Eq. 2: log det not doubled",
     [PINS], "  logdet *= 2.0;\n  oracle_forward_solve", "  oracle_forward_solve", 1),
    ("Eq. 3: sign of ln 2 in log c",
     [PINS], "(1.0 - nu) * ORACLE_LN2 - lgamma(nu);\n  return sigma2",
     "(nu - 1.0) * ORACLE_LN2 - lgamma(nu);\n  return sigma2", 1),
    ("Eq. 3: Euclidean distance not square-rooted",
     [PINS], "return sqrt(dx * dx + dy * dy);", "return dx * dx + dy * dy;", 1),
    ("K_nu: full weight at the trapezoid's t = 0 node",
     [PINS], "double sum = 0.5;", "double sum = 1.0;", 1),
    ("K_nu: cosh(t) in place of cosh(nu t)",
     [PINS], "exp(-x * 2.0 * sh * sh) * cosh(nu * t)", "exp(-x * 2.0 * sh * sh) * cosh(t)", 1),
    ("dK/dnu: cosh in place of sinh",
     [PINS], "t * sinh(nu * t) * exp", "t * cosh(nu * t) * exp", 1),
    ("digamma: wrong sign in the recurrence",
     [PINS], "acc -= 1.0 / x;", "acc += 1.0 / x;", 1),
    ("digamma: sign of B_4 / 4",
     [PINS], "x2 * (-1.0 / 120.0 +", "x2 * (1.0 / 120.0 +", 1),
    ("dSigma/dbeta: K_{nu+1} in place of K_{nu-1}",
     [PINS], "oracle_besselk_scaled(nu - 1.0, x) * x / beta", "oracle_besselk_scaled(nu + 1.0, x) * x / beta", 1),
    ("dSigma/dnu: sign of psi",
     [PINS], "-ORACLE_LN2 - oracle_digamma(nu) + log(x)", "-ORACLE_LN2 + oracle_digamma(nu) + log(x)", 1),
    ("gradient: sign of the trace term",
     [PINS], "grad[c] = 0.5 * quadform - 0.5 * trace;", "grad[c] = 0.5 * quadform + 0.5 * trace;", 1),
    ("gradient: Sigma^-1 = X^T X summed from the wrong row",
     [PINS, FISHER], "for (int64_t k = i; k < n; ++k) t += X[k * n + i] * X[k * n + j];",
     "for (int64_t k = i + 1; k < n; ++k) t += X[k * n + i] * X[k * n + j];", 2),
    ("back solve: transposed index",
     [PINS], "t -= L[k * n + i] * a[k];", "t -= L[i * n + k] * a[k];", 1),
    ("Cholesky: column not divided by the pivot",
     [PINS], "Li[j] = t / ljj;", "Li[j] = t;", 1),
    ("Cholesky: pivot without its square root",
     [PINS], "const double ljj = sqrt(s);", "const double ljj = s;", 1),
    ("forward solve: inner sum one term short",
     [PINS], "for (int64_t k = 0; k < i; ++k) t -= Li[k] * y[k];",
     "for (int64_t k = 0; k + 1 < i; ++k) t -= Li[k] * y[k];", 1),
    ("great circle: full angle in the haversine",
     [MODEL], "sin(0.5 * (p2 - p1))", "sin(p2 - p1)", 1),
    ("nugget added off the diagonal",
     [MODEL], "oracle_dist(locs, i, j)) + (i == j ? g_nugget : 0.0);", "oracle_dist(locs, i, j)) + g_nugget;", 1),
    ("great circle: latitude and longitude swapped",
     [MODEL], "const double p1 = y1 * rad, p2 = y2 * rad;\n    const double sp = sin(0.5 * (p2 - p1)), "
              "sl = sin(0.5 * (x2 - x1) * rad);",
     "const double p1 = x1 * rad, p2 = x2 * rad;\n    const double sp = sin(0.5 * (p2 - p1)), "
     "sl = sin(0.5 * (y2 - y1) * rad);", 1),
    ("nugget dropped",
     [MODEL], "oracle_dist(locs, i, j)) + (i == j ? g_nugget : 0.0);", "oracle_dist(locs, i, j));", 1),
    ("kriging: variance reduction halved",
     [PREDICT], "var[i] = theta[0] - ww;", "var[i] = theta[0] - 0.5 * ww;", 1),
    ("kriging: sign of the variance reduction",
     [PREDICT], "var[i] = theta[0] - ww;", "var[i] = theta[0] + ww;", 1),
    ("kriging: mean from L^-1 Z instead of Sigma^-1 Z",
     [PREDICT], "mu += c[j] * a[j];", "mu += c[j] * y[j];", 1),
    ("Fisher: the 1/2 dropped",
     [FISHER], "out[k * 3 + l] = 0.5 * t;", "out[k * 3 + l] = t;", 1),
    ("Fisher: M_l not transposed in the trace",
     [FISHER], "t += Mk[i * n + j] * Ml[j * n + i];", "t += Mk[i * n + j] * Ml[i * n + j];", 1),
]

RUNNER = """
import sys
tmp, files = sys.argv[1], sys.argv[2:]
sys.path.insert(0, tmp)
import oracle
assert oracle.__file__.startswith(tmp), oracle.__file__
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + files))
"""


def _run_with(tmp_path, mutate):
    """Copy oracle/, apply `mutate` to oracle.c, compile it, run the runner; returns (rc, output tail)."""
    dst = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    src = dst / "oracle.c"
    src.write_text(mutate(src.read_text()))
    (dst / "_build").mkdir()
    # compiled here, with the flags the oracle uses, so a mutant that fails to build cannot pass for a caught one
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o",
                           str(dst / "_build" / "liboracle.so"), str(src), "-lm"])
    return _runner(tmp_path, mutate.files)


def _runner(tmp_path, files):
    env = dict(os.environ, OMP_NUM_THREADS="4", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-c", RUNNER, str(tmp_path)] + list(files), cwd=str(tmp_path), env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


class _Mutation:
    def __init__(self, old, new, count, files):
        self.old, self.new, self.count, self.files = old, new, count, files

    def __call__(self, text):
        assert text.count(self.old) == self.count, "mutation target not found as expected: %r" % self.old
        return text.replace(self.old, self.new)


def test_unmutated_copy_passes_its_pins(tmp_path):
    rc, out = _run_with(tmp_path, _Mutation("#include <math.h>", "#include <math.h>", 1, [PINS, MODEL, PREDICT, FISHER]))
    assert rc == 0, out


@pytest.mark.parametrize("name,files,old,new,count", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, files, old, new, count):
    rc, out = _run_with(tmp_path, _Mutation(old, new, count, files))
    # 1 = some test failed; 0 would mean the pins missed the mistake, >1 a collection or internal error
    assert rc == 1, "%s: pytest exit code %d\n%s" % (name, rc, out)
