"""Pins for the FP64 oracle: checks against what the paper and mathematics fix.

Each test compares the oracle with something other than itself: closed forms
(the exponential special case the paper names under Eq. 3, the half-integer
spherical-Bessel forms, the n = 1 and n = 2 likelihoods), textbook identities,
independent libraries (mpmath, scipy, numpy LAPACK), brute-force elimination
on tiny inputs and exact invariants of Eq. 2.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth

XS = [1e-6, 1e-3, 0.01, 0.1, 0.5, 1.0, 1.9, 2.0, 2.1, 3.0, 7.5, 20.0, 60.0, 250.0, 700.0]
NUS = [0.1, 0.25, 0.5, 0.73, 1.0, 1.37, 1.5, 2.0, 2.5]


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# --- K_nu --------------------------------------------------------------------

@pytest.mark.parametrize("x", XS)
def test_besselk_half_integer_closed_forms(x):
    # DLMF 10.39.2 / 10.49.12: K_{1/2}, K_{3/2}, K_{5/2} in elementary form
    base = math.sqrt(math.pi / (2 * x))
    assert rel(oracle.besselk_scaled(0.5, x), base) < 2e-15
    assert rel(oracle.besselk_scaled(1.5, x), base * (1 + 1 / x)) < 2e-15
    assert rel(oracle.besselk_scaled(2.5, x), base * (1 + 3 / x + 3 / x**2)) < 2e-15


@pytest.mark.parametrize("nu", NUS)
def test_besselk_recurrence_and_evenness(nu):
    # DLMF 10.29.1: K_{nu+1} = K_{nu-1} + (2 nu / x) K_nu ;  K_{-nu} = K_nu
    for x in [0.05, 0.7, 2.0, 5.0, 40.0]:
        lhs = oracle.besselk_scaled(nu + 1, x)
        rhs = oracle.besselk_scaled(nu - 1, x) + 2 * nu / x * oracle.besselk_scaled(nu, x)
        assert rel(lhs, rhs) < 1e-14
        assert oracle.besselk_scaled(-nu, x) == oracle.besselk_scaled(nu, x)


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.5, 2.0])
def test_matern_small_distance_limit(nu):
    # x^nu K_nu(x) -> 2^(nu-1) Gamma(nu) as x -> 0, i.e. Sigma_ij -> sigma^2
    th = [2.5, 0.1, nu]
    assert rel(oracle.matern(th, 1e-9), 2.5) < 1e-6


@pytest.mark.parametrize("nu", NUS)
def test_matern_decreasing_and_within_sigma2(nu):
    # d/dx [x^nu K_nu(x)] = -x^nu K_{nu-1}(x) < 0 (DLMF 10.29.4) and x^nu K_nu(x) -> 2^(nu-1) Gamma(nu)
    # as x -> 0: Eq. 3 falls strictly from sigma^2 towards 0 as the distance grows
    th = [1.7, 0.2, nu]
    r = np.geomspace(1e-6, 12.0, 400)  # x = r / beta from 5e-6 to 60
    v = np.array([oracle.matern(th, float(t)) for t in r])
    assert np.all(v > 0.0) and np.all(v <= 1.7 * (1 + 1e-15))
    assert np.all(np.diff(v) < 0.0)
    assert oracle.matern(th, 0.0) == 1.7


def test_besselk_vs_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for nu in NUS + [0.0, 0.999999, 1.000001]:
        for x in XS:
            ref = float(mp.besselk(nu, x) * mp.exp(x))
            assert rel(oracle.besselk_scaled(nu, x), ref) < 2e-15, (nu, x)


def test_besselk_vs_scipy():
    sp = pytest.importorskip("scipy.special")
    for nu in NUS:
        for x in XS:
            assert rel(oracle.besselk_scaled(nu, x), sp.kve(nu, x)) < 2e-13, (nu, x)


def test_dbesselk_dnu_closed_form_half():
    # DLMF 10.38.7: dK_nu/dnu at nu = 1/2 is sqrt(pi/(2x)) E_1(2x) e^x
    sp = pytest.importorskip("scipy.special")
    for x in [1e-3, 0.02, 0.3, 1.0, 2.0, 6.0, 30.0, 200.0]:
        ref = math.sqrt(math.pi / (2 * x)) * sp.exp1(2 * x) * math.exp(x)
        assert rel(oracle.dbesselk_dnu(0.5, x), ref) < 2e-14, x


def test_dbesselk_dnu_zero_at_nu_zero_and_odd():
    for x in [0.1, 1.0, 10.0]:
        assert oracle.dbesselk_dnu(0.0, x) == 0.0
        assert rel(oracle.dbesselk_dnu(-0.7, x), -oracle.dbesselk_dnu(0.7, x)) < 1e-15


def test_dbesselk_dnu_vs_mpmath_derivative():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for nu in [0.1, 0.73, 1.0, 1.5, 2.0]:
        for x in [1e-3, 0.05, 0.9, 2.0, 4.5, 25.0]:
            ref = float(mp.diff(lambda v: mp.besselk(v, x), nu))
            assert rel(oracle.dbesselk_dnu(nu, x), ref) < 5e-14, (nu, x)


def test_digamma_special_values():
    gamma_e = 0.57721566490153286061
    assert abs(oracle.digamma(1.0) + gamma_e) < 1e-15
    assert abs(oracle.digamma(0.5) + gamma_e + 2 * math.log(2)) < 1e-15
    for x in [0.1, 0.9, 3.3, 12.0]:
        assert abs(oracle.digamma(x + 1) - oracle.digamma(x) - 1 / x) < 1e-13
    # psi(n) = H_{n-1} - gamma
    for n in [2, 5, 11]:
        assert abs(oracle.digamma(n) - (sum(1.0 / k for k in range(1, n)) - gamma_e)) < 1e-14


# --- Matérn covariance (Eq. 3) ----------------------------------------------

@pytest.mark.parametrize("r", [1e-4, 0.01, 0.05, 0.2, 0.7, 1.4])
def test_matern_exponential_special_case(r):
    # Section I (under Eq. 3): nu = 1/2 is the exponential kernel sigma^2 exp(-r/beta)
    for s2, beta in [(1.0, 0.1), (0.3, 0.03), (4.0, 1.7)]:
        th = [s2, beta, 0.5]
        ref = s2 * math.exp(-r / beta)
        # exp(-x) amplifies the rounding of its argument: allow ~ulp(x) relative
        tol = 3e-15 + 2.5e-16 * (r / beta)
        assert rel(oracle.matern(th, r), ref) < tol
        assert rel(oracle.matern_direct(th, r), ref) < 10 * tol


@pytest.mark.parametrize("r", [1e-3, 0.05, 0.3, 1.2])
def test_matern_higher_half_integers(r):
    # nu = 3/2: sigma^2 (1 + x) e^-x ; nu = 5/2: sigma^2 (1 + x + x^2/3) e^-x, x = r/beta
    for beta in [0.03, 0.1, 0.6]:
        x = r / beta
        tol = 4e-15 + 2.5e-16 * x
        assert rel(oracle.matern([1.3, beta, 1.5], r), 1.3 * (1 + x) * math.exp(-x)) < tol
        assert rel(oracle.matern([1.3, beta, 2.5], r), 1.3 * (1 + x + x * x / 3) * math.exp(-x)) < tol


def test_matern_log_and_direct_forms_agree():
    for nu in [0.3, 1.0, 1.8]:
        for r in [0.002, 0.05, 0.4]:
            th = [1.1, 0.13, nu]
            assert rel(oracle.matern(th, r), oracle.matern_direct(th, r)) < 1e-13


def test_matern_grad_vs_finite_differences():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for th in ([1.0, 0.1, 0.5], [1.5, 0.2, 1.5], [0.7, 0.05, 1.0], [2.0, 0.3, 0.37]):
        for r in [0.003, 0.04, 0.25, 0.9]:
            g = oracle.matern_grad(th, r)

            def f(s2, b, v):
                x = mp.mpf(r) / b
                return s2 * 2 ** (1 - v) / mp.gamma(v) * x**v * mp.besselk(v, x)

            ref = [float(mp.diff(lambda s: f(s, th[1], th[2]), th[0])),
                   float(mp.diff(lambda b: f(th[0], b, th[2]), th[1])),
                   float(mp.diff(lambda v: f(th[0], th[1], v), th[2]))]
            # d/dnu is a difference of terms of size sigma^2 (1 + |ln x|): bound the error by that scale
            scale = [abs(ref[0]), abs(ref[1]), th[0] * (1 + abs(math.log(r / th[1]))) + abs(ref[2])]
            for c in range(3):
                assert abs(g[c] - ref[c]) <= 1e-13 * max(scale[c], 1e-30) + 1e-300, (th, r, c)
    assert list(oracle.matern_grad([1.0, 0.1, 0.5], 0.0)) == [1.0, 0.0, 0.0]


def test_covariance_symmetric_spd():
    locs = synth.jittered_grid(8, seed=3)
    for th in ([1.0, 0.1, 0.5], [1.5, 0.2, 1.5], [1.0, 0.03, 1.0]):
        S = oracle.covariance(locs, th)
        assert np.array_equal(S, S.T)
        assert np.all(np.diag(S) == th[0])
        L, info = oracle.cholesky(S)
        assert info == 0 and np.all(np.diag(L) > 0)
        assert np.max(np.abs(L @ L.T - S)) < 1e-14 * th[0] * 64


def test_covariance_entries_match_full():
    locs = synth.jittered_grid(6, seed=4)
    th = [1.0, 0.1, 0.5]
    S = oracle.covariance(locs, th)
    rows = np.array([0, 5, 35, 17, 3])
    cols = np.array([0, 2, 1, 17, 30])
    assert np.array_equal(oracle.covariance_entries(locs, th, rows, cols), S[rows, cols])


# --- log-likelihood (Eq. 2) --------------------------------------------------

def test_loglik_n1_closed_form():
    for s2 in [0.5, 1.0, 3.0]:
        for z in [-1.3, 0.0, 2.2]:
            r = oracle.loglik([[0.3, 0.4]], [z], [s2, 0.1, 0.5])
            ref = -0.5 * math.log(2 * math.pi) - 0.5 * math.log(s2) - z * z / (2 * s2)
            assert abs(r["l"] - ref) < 1e-15 * 4


def test_loglik_n2_closed_form():
    for nu in [0.5, 1.0, 1.7]:
        locs = [[0.1, 0.2], [0.15, 0.26]]
        th = [1.7, 0.09, nu]
        z1, z2 = 0.8, -0.35
        rho = oracle.matern(th, math.hypot(0.05, 0.06)) / th[0]
        s2 = th[0]
        ref = (-math.log(2 * math.pi) - 0.5 * math.log(s2 * s2 * (1 - rho * rho))
               - (z1 * z1 - 2 * rho * z1 * z2 + z2 * z2) / (2 * s2 * (1 - rho * rho)))
        r = oracle.loglik(locs, [z1, z2], th)
        assert rel(r["l"], ref) < 1e-14


def _lu_brute(A):
    """Gaussian elimination with partial pivoting, pure Python: (log|det|, sign, LU, perm)."""
    A = [list(map(float, row)) for row in A]
    n = len(A)
    perm = list(range(n))
    logdet, sign = 0.0, 1.0
    for k in range(n):
        p = max(range(k, n), key=lambda i: abs(A[i][k]))
        if p != k:
            A[k], A[p] = A[p], A[k]
            perm[k], perm[p] = perm[p], perm[k]
            sign = -sign
        piv = A[k][k]
        logdet += math.log(abs(piv))
        sign *= 1 if piv > 0 else -1
        for i in range(k + 1, n):
            f = A[i][k] / piv
            A[i][k] = f
            for j in range(k + 1, n):
                A[i][j] -= f * A[k][j]
    return logdet, sign, A, perm


def _lu_solve(LU, perm, b):
    n = len(LU)
    y = [b[perm[i]] for i in range(n)]
    for i in range(n):
        for k in range(i):
            y[i] -= LU[i][k] * y[k]
    for i in reversed(range(n)):
        for k in range(i + 1, n):
            y[i] -= LU[i][k] * y[k]
        y[i] /= LU[i][i]
    return y


@pytest.mark.parametrize("m,th", [(3, [1.0, 0.1, 0.5]), (5, [1.5, 0.2, 1.5]), (8, [1.0, 0.03, 1.0]),
                                  (8, [0.6, 0.4, 0.8])])
def test_loglik_vs_bruteforce_lu(m, th):
    locs = synth.jittered_grid(m, seed=m)
    n = m * m
    Z = synth.normals(n, seed=m)
    S = oracle.covariance(locs, th)
    logdet, sign, LU, perm = _lu_brute(S)
    assert sign == 1.0
    x = _lu_solve(LU, perm, list(Z))
    quad = float(np.dot(Z, x))
    r = oracle.loglik(locs, Z, th)
    assert rel(r["logdet"], logdet) < 1e-12
    assert rel(r["quad"], quad) < 1e-12
    ref = -0.5 * n * math.log(2 * math.pi) - 0.5 * logdet - 0.5 * quad
    assert rel(r["l"], ref) < 1e-12
    # and against LAPACK through numpy
    s_np, ld_np = np.linalg.slogdet(S)
    assert s_np == 1.0 and rel(r["logdet"], ld_np) < 1e-12
    assert rel(r["quad"], float(Z @ np.linalg.solve(S, Z))) < 1e-11


def test_loglik_coincident_points_singular():
    # Section III (Example 2): Sigma is singular when two locations coincide; the pivot of the
    # duplicate collapses to rounding level (it may land on either side of zero)
    locs = synth.jittered_grid(4, seed=1)
    locs[7] = locs[3]
    S = oracle.covariance(locs, [1.0, 0.1, 0.5])
    L, info = oracle.cholesky(S)
    assert info == 8 or (info == 0 and L[7, 7] ** 2 < 1e-13)


def test_loglik_not_spd_nan_location():
    locs = synth.jittered_grid(4, seed=1)
    locs[5, 0] = float("nan")
    r = oracle.loglik(locs, synth.normals(16, 1), [1.0, 0.1, 0.5])
    assert r["info"] == 6 and math.isnan(r["l"])


def test_invariant_sigma2_scaling():
    # l(sigma^2) = -(n/2) ln 2pi - (n/2) ln sigma^2 - 1/2 log|R| - q_R / (2 sigma^2)
    locs = synth.jittered_grid(7, seed=2)
    Z = synth.normals(49, 2)
    base = oracle.loglik(locs, Z, [1.0, 0.15, 1.3])
    n = 49
    for s2 in [0.2, 2.7]:
        r = oracle.loglik(locs, Z, [s2, 0.15, 1.3])
        ref = -0.5 * n * math.log(2 * math.pi) - 0.5 * n * math.log(s2) - 0.5 * base["logdet"] - base["quad"] / (2 * s2)
        assert rel(r["l"], ref) < 1e-13


def test_invariant_permutation_translation_scaling():
    locs = synth.jittered_grid(6, seed=5)
    Z = synth.normals(36, 5)
    th = [1.2, 0.2, 0.9]
    base = oracle.loglik(locs, Z, th)["l"]
    perm = np.random.default_rng(0).permutation(36)
    assert rel(oracle.loglik(locs[perm], Z[perm], th)["l"], base) < 1e-12
    assert rel(oracle.loglik(locs + np.array([3.25, -1.5]), Z, th)["l"], base) < 1e-10
    assert rel(oracle.loglik(locs * 4.0, Z, [1.2, 0.8, 0.9])["l"], base) < 1e-12


def test_invariant_independence_limit():
    # beta tiny: off-diagonal entries vanish and l = -(n/2) ln(2 pi sigma^2) - |Z|^2 / (2 sigma^2)
    locs = synth.jittered_grid(10, seed=6)
    Z = synth.normals(100, 6)
    s2 = 1.7
    r = oracle.loglik(locs, Z, [s2, 1e-4, 1.0])
    ref = -50 * math.log(2 * math.pi * s2) - float(Z @ Z) / (2 * s2)
    assert rel(r["l"], ref) < 1e-14


def test_invariant_block_diagonal():
    a = synth.jittered_grid(4, seed=7)
    b = synth.jittered_grid(5, seed=8) + 50.0
    Za, Zb = synth.normals(16, 7), synth.normals(25, 8)
    th = [1.0, 0.1, 1.5]
    la = oracle.loglik(a, Za, th)["l"]
    lb = oracle.loglik(b, Zb, th)["l"]
    lab = oracle.loglik(np.vstack([a, b]), np.concatenate([Za, Zb]), th)["l"]
    assert rel(lab, la + lb) < 1e-13


# --- gradient ------------------------------------------------------------------

@pytest.mark.parametrize("th", [[1.0, 0.1, 0.5], [1.5, 0.2, 1.5], [0.8, 0.05, 1.0]])
def test_gradient_sigma2_closed_form_and_fd(th):
    locs = synth.jittered_grid(6, seed=9)
    n = 36
    Z = synth.normals(n, 9)
    g = oracle.loglik_grad(locs, Z, th)
    assert g["info"] == 0
    assert rel(g["l"], oracle.loglik(locs, Z, th)["l"]) < 1e-14
    # Sigma is proportional to sigma^2, so dl/dsigma^2 = (Z^T Sigma^-1 Z - n) / (2 sigma^2)
    s2 = th[0]
    assert rel(g["grad"][0], (g["quad"] - n) / (2 * s2)) < 1e-10
    # central differences, Richardson-extrapolated
    for c in range(3):
        def l_at(d):
            t = list(th)
            t[c] += d
            return oracle.loglik(locs, Z, t)["l"]
        h = 1e-3 * th[c]
        d1 = (l_at(h) - l_at(-h)) / (2 * h)
        d2 = (l_at(h / 2) - l_at(-h / 2)) / h
        fd = (4 * d2 - d1) / 3
        assert abs(g["grad"][c] - fd) <= 2e-7 * max(1.0, abs(fd)), (c, g["grad"][c], fd)


def test_gradient_zero_at_profile_sigma2():
    # the profile maximiser in sigma^2 is q_R / n, where dl/dsigma^2 = 0
    locs = synth.jittered_grid(5, seed=10)
    Z = synth.normals(25, 10)
    base = oracle.loglik(locs, Z, [1.0, 0.2, 1.0])
    s2hat = base["quad"] / 25
    g = oracle.loglik_grad(locs, Z, [s2hat, 0.2, 1.0])
    assert abs(g["grad"][0]) < 1e-12 * 25 / s2hat


def test_simulate_matches_lapack_factor():
    locs = synth.jittered_grid(6, seed=11)
    th = [1.0, 0.1, 0.5]
    eps = synth.normals(36, 11)
    Z = oracle.simulate(locs, th, eps)
    Lnp = np.linalg.cholesky(oracle.covariance(locs, th))
    assert np.max(np.abs(Z - Lnp @ eps)) < 1e-13
