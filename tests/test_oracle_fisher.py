"""Pins for the oracle's Fisher information I_kl = 1/2 tr(Sigma^-1 D_k Sigma^-1 D_l) (exact_fisher):
the sigma^2 closed form, the exponential case with closed-form derivatives, finite differences of
Sigma, symmetry and positive definiteness, and the score-covariance identity I = E[g g^T]."""
import math

import numpy as np

import oracle
from paper_1908_06936_gb300 import synth


def test_sigma2_entry_closed_form():
    # D_sigma2 = Sigma / sigma^2, so Sigma^-1 D = I / sigma^2 and I_11 = n / (2 sigma^4)
    for th in [(2.0, 0.1, 0.7), (0.5, 0.3, 1.6)]:
        locs = synth.jittered_grid(6, 4)
        F = oracle.fisher(locs, th)
        assert abs(F[0, 0] - 36 / (2 * th[0] ** 2)) <= 1e-12 * F[0, 0]


def test_exponential_case_closed_form_derivatives():
    # nu = 1/2: Sigma = s exp(-r/b), dSigma/ds = exp(-r/b), dSigma/db = s r/b^2 exp(-r/b)
    th = (1.4, 0.12, 0.5)
    locs = synth.jittered_grid(5, 6)
    R = np.sqrt(((locs[:, None, :] - locs[None, :, :]) ** 2).sum(-1))
    E = np.exp(-R / th[1])
    S = th[0] * E
    Si = np.linalg.inv(S)
    D = [E, th[0] * R / th[1] ** 2 * E]
    F = oracle.fisher(locs, th)
    for k in range(2):
        for l in range(2):
            ref = 0.5 * np.trace(Si @ D[k] @ Si @ D[l])
            assert abs(F[k, l] - ref) <= 1e-9 * abs(ref), (k, l, F[k, l], ref)


def test_vs_finite_differences_of_sigma():
    th = np.array([1.1, 0.15, 1.3])
    locs = synth.jittered_grid(5, 7)
    Si = np.linalg.inv(oracle.covariance(locs, th))
    D = []
    for k in range(3):
        h = 1e-5 * th[k]
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        D.append((oracle.covariance(locs, tp) - oracle.covariance(locs, tm)) / (2 * h))
    ref = np.array([[0.5 * np.trace(Si @ D[k] @ Si @ D[l]) for l in range(3)] for k in range(3)])
    F = oracle.fisher(locs, th)
    assert np.allclose(F, ref, rtol=1e-6, atol=0), np.max(np.abs(F - ref) / np.abs(ref))


def test_symmetric_positive_definite():
    F = oracle.fisher(synth.jittered_grid(6, 9), (1.0, 0.2, 0.9))
    assert np.allclose(F, F.T, rtol=1e-12, atol=0)
    assert np.all(np.linalg.eigvalsh(F) > 0)


def test_score_covariance_identity():
    # I = E[g g^T] for the score g = dl/dtheta at the true theta (Z ~ N(0, Sigma))
    th = (1.0, 0.25, 0.8)
    locs = synth.jittered_grid(3, 11)
    N = 20000
    rng = np.random.default_rng(0)
    L = np.linalg.cholesky(oracle.covariance(locs, th))
    G = np.empty((N, 3))
    for s in range(N):
        G[s] = oracle.loglik_grad(locs, L @ rng.standard_normal(9), th)["grad"]
    emp = G.T @ G / N
    F = oracle.fisher(locs, th)
    # each entry of the sample average has relative standard error ~ sqrt(2 / N) ~ 1%
    assert np.all(np.abs(emp - F) <= 0.06 * np.sqrt(np.outer(np.diag(F), np.diag(F)))), (emp, F)
