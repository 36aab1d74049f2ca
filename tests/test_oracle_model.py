"""Pins for the oracle's model options (the paper's dmetric and a nugget): great-circle
distances of known geometry, rotation invariance, and the nugget's closed-form likelihoods."""
import math

import numpy as np
import pytest

import oracle
from paper_1908_06936_gb300 import synth

R = 6371.0


@pytest.fixture(autouse=True)
def reset_model():
    yield
    oracle.set_model()


def gc_dist_via_cov(p, q, radius=R):
    # nu = 1/2, sigma^2 = 1, beta = 1: Sigma_12 = exp(-d)  ->  d = -ln Sigma_12
    oracle.set_model(0.0, 1, radius)
    S = oracle.covariance(np.array([p, q], dtype=float), (1.0, 1.0, 0.5))
    return -math.log(S[0, 1])


@pytest.mark.parametrize("p,q,d", [((0, 0), (90, 0), math.pi / 2), ((10, 90), (77, 0), math.pi / 2),
                                   ((0, 0), (180, 0), math.pi), ((25, -30), (205, 30), math.pi),
                                   ((0, 0), (0, 1), math.pi / 180)])
def test_great_circle_known_distances(p, q, d):
    radius = 10.0  # keeps exp(-d) representable
    assert abs(gc_dist_via_cov(p, q, radius) - radius * d) <= 1e-12 * radius * d


def test_great_circle_small_arc_along_a_parallel():
    # at latitude phi a small longitude step dl spans ~ R cos(phi) dl
    for phi in (0.0, 45.0, 60.0):
        dl = 1e-3
        d = gc_dist_via_cov((5.0, phi), (5.0 + dl, phi), radius=1.0)
        assert abs(d - math.cos(math.radians(phi)) * math.radians(dl)) <= 1e-9 * d


def test_great_circle_rotation_invariance_and_symmetry():
    oracle.set_model(0.0, 1, R)
    rng = np.random.default_rng(3)
    locs = np.column_stack([rng.uniform(-180, 180, 30), rng.uniform(-70, 70, 30)])
    th = (1.0, 800.0, 1.3)
    S1 = oracle.covariance(locs, th)
    shifted = locs.copy()
    shifted[:, 0] = (shifted[:, 0] + 37.0 + 180.0) % 360.0 - 180.0
    S2 = oracle.covariance(shifted, th)
    assert np.allclose(S1, S2, rtol=1e-10, atol=1e-14)
    assert np.allclose(S1, S1.T, rtol=0, atol=0)
    assert np.all(np.linalg.eigvalsh(S1) > 0)


def test_nugget_on_the_diagonal_only():
    locs = synth.jittered_grid(5, 2)
    th = (1.3, 0.1, 0.8)
    S0 = oracle.covariance(locs, th)
    oracle.set_model(0.25, 0, R)
    S1 = oracle.covariance(locs, th)
    assert np.allclose(np.diag(S1), th[0] + 0.25, rtol=1e-15, atol=0)
    assert np.array_equal(S1 - np.diag(np.diag(S1)), S0 - np.diag(np.diag(S0)))


def test_nugget_closed_form_likelihoods():
    th, tau2 = (1.5, 0.2, 0.5), 0.3
    oracle.set_model(tau2, 0, R)
    z1 = np.array([0.7])
    v = th[0] + tau2
    l1 = oracle.loglik(np.array([[0.2, 0.4]]), z1, th)["l"]
    assert abs(l1 - (-0.5 * math.log(2 * math.pi * v) - 0.5 * z1[0] ** 2 / v)) <= 1e-14
    locs = np.array([[0.1, 0.1], [0.25, 0.3]])
    z = np.array([0.4, -1.1])
    c = th[0] * math.exp(-math.dist(locs[0], locs[1]) / th[1])
    det = v * v - c * c
    quad = (v * z[0] ** 2 - 2 * c * z[0] * z[1] + v * z[1] ** 2) / det
    l2 = oracle.loglik(locs, z, th)["l"]
    assert abs(l2 - (-math.log(2 * math.pi) - 0.5 * math.log(det) - 0.5 * quad)) <= 1e-13


def test_nugget_regularises_coincident_points():
    locs = synth.jittered_grid(4, 1)
    locs[3] = locs[2]
    th = (1.0, 0.3, 1.5)
    oracle.set_model(0.1, 0, R)
    r = oracle.loglik(locs, synth.normals(16, 1), th)
    assert r["info"] == 0 and math.isfinite(r["l"])
