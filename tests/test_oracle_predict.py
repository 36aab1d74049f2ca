"""Pins for the oracle's kriging (spatial prediction at new locations, the conditional
Gaussian mean and variance of Section IV's exact_predict), checked against what the
mathematics fixes: interpolation at observed points, the one-point closed form, the
far-field limit, the joint-precision formula by brute-force elimination, linearity and
scaling."""
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth
from test_oracle_pins import _lu_brute, _lu_solve


def expo(theta, r):
    # nu = 1/2: Eq. 3 reduces to sigma^2 exp(-r / beta)
    return theta[0] * math.exp(-r / theta[1])


def test_interpolates_observed_points():
    th = (1.3, 0.1, 0.5)
    locs = synth.jittered_grid(7, 2)
    z = synth.normals(49, 2)
    idx = [0, 5, 17, 48]
    mean, var = oracle.predict(locs, z, th, locs[idx])
    assert np.allclose(mean, z[idx], rtol=0, atol=1e-10)
    assert np.all(np.abs(var) <= 1e-10 * th[0])


@pytest.mark.parametrize("r", [0.01, 0.07, 0.3])
def test_single_observation_closed_form(r):
    th = (2.0, 0.1, 0.5)
    locs = np.array([[0.2, 0.3]])
    new = np.array([[0.2 + r * 0.6, 0.3 + r * 0.8]])
    z = np.array([1.7])
    mean, var = oracle.predict(locs, z, th, new)
    rho = math.exp(-r / th[1])
    assert abs(mean[0] - rho * z[0]) <= 1e-13 * abs(z[0])
    assert abs(var[0] - th[0] * (1.0 - rho * rho)) <= 1e-13 * th[0]


def test_far_field_limit():
    th = (1.0, 0.01, 1.0)
    locs = synth.jittered_grid(5, 3) * 0.2
    z = synth.normals(25, 3)
    mean, var = oracle.predict(locs, z, th, np.array([[0.95, 0.95]]))  # r / beta >= 100
    assert abs(mean[0]) <= 1e-30 and abs(var[0] - th[0]) <= 1e-15


@pytest.mark.parametrize("m,th", [(3, (1.0, 0.1, 0.5)), (4, (0.7, 0.25, 0.5))])
def test_joint_precision_formula_by_elimination(m, th):
    # x = (obs, new) jointly Gaussian with covariance J; with P = J^-1:
    #   Var(new | obs) = 1 / P_nn,  E(new | obs) = -(P_no z) / P_nn
    locs = synth.jittered_grid(m, m)
    n = m * m
    z = synth.normals(n, m)
    new = np.array([[0.37, 0.61]])
    pts = np.vstack([locs, new])
    J = [[expo(th, math.dist(pts[i], pts[j])) for j in range(n + 1)] for i in range(n + 1)]
    _, _, LU, perm = _lu_brute(J)
    e = [0.0] * (n + 1)
    e[n] = 1.0
    p = _lu_solve(LU, perm, e)  # column n of P (P symmetric)
    var_ref = 1.0 / p[n]
    mean_ref = -sum(p[j] * z[j] for j in range(n)) / p[n]
    mean, var = oracle.predict(locs, z, th, new)
    assert abs(var[0] - var_ref) <= 1e-11 * th[0]
    assert abs(mean[0] - mean_ref) <= 1e-11 * max(1.0, abs(mean_ref))


def test_linear_in_data_and_scaling():
    th = (1.0, 0.15, 1.2)
    locs = synth.jittered_grid(6, 8)
    z1, z2 = synth.normals(36, 8), synth.normals(36, 9)
    new = synth.uniform_square(10, 4)
    m1, v1 = oracle.predict(locs, z1, th, new)
    m2, v2 = oracle.predict(locs, z2, th, new)
    m3, v3 = oracle.predict(locs, 2.0 * z1 - 0.5 * z2, th, new)
    assert np.allclose(m3, 2.0 * m1 - 0.5 * m2, rtol=1e-12, atol=1e-12)
    assert np.allclose(v1, v2, rtol=0, atol=1e-14) and np.allclose(v1, v3, rtol=0, atol=1e-14)
    # sigma^2 cancels in the mean and scales the variance
    m4, v4 = oracle.predict(locs, z1, (3.0, th[1], th[2]), new)
    assert np.allclose(m4, m1, rtol=1e-11, atol=1e-13)
    assert np.allclose(v4, 3.0 * v1, rtol=1e-10, atol=1e-14)
    assert np.all(v1 > 0) and np.all(v1 < th[0])
