"""FP64 CPU oracle for the exact Matérn Gaussian log-likelihood.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this package; the product path (the
CUDA library and its binding) never does and shares no code with it.

The C source ``oracle.c`` writes out the paper's definitions: Eq. 2 (Gaussian
log-likelihood, zero mean), Eq. 3 (Matérn covariance) and the Cholesky-based
evaluation of Section I.  This module compiles it with gcc (OpenMP) on first
use and exposes numpy-friendly wrappers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain gcc, no -ffast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "oracle_besselk": (_D, [_D, _D]),
                "oracle_besselk_scaled": (_D, [_D, _D]),
                "oracle_dbesselk_dnu": (_D, [_D, _D]),
                "oracle_dbesselk_dnu_scaled": (_D, [_D, _D]),
                "oracle_digamma": (_D, [_D]),
                "oracle_matern": (_D, [_PD, _D]),
                "oracle_matern_direct": (_D, [_PD, _D]),
                "oracle_matern_grad": (None, [_PD, _D, _PD]),
                "oracle_covariance": (None, [_I64, _PD, _PD, _PD]),
                "oracle_covariance_entries": (None, [_I64, _PI64, _PI64, _PD, _PD, _PD]),
                "oracle_cholesky": (_I64, [_I64, _PD]),
                "oracle_forward_solve": (None, [_I64, _PD, _PD, _PD]),
                "oracle_backward_solve": (None, [_I64, _PD, _PD, _PD]),
                "oracle_loglik": (_I64, [_I64, _PD, _PD, _PD, _PD]),
                "oracle_loglik_grad": (_I64, [_I64, _PD, _PD, _PD, _PD, _PD]),
                "oracle_simulate": (_I64, [_I64, _PD, _PD, _PD, _PD]),
                "oracle_predict": (_I64, [_I64, _PD, _PD, _PD, _I64, _PD, _PD, _PD]),
                "oracle_fisher": (_I64, [_I64, _PD, _PD, _PD]),
                "oracle_set_model": (None, [_D, ctypes.c_int, _D]),
                "oracle_max_threads": (ctypes.c_int, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def besselk(nu: float, x: float) -> float:
    """K_nu(x) by trapezoidal quadrature of DLMF 10.32.9."""
    return _load().oracle_besselk(float(nu), float(x))


def besselk_scaled(nu: float, x: float) -> float:
    """e^x K_nu(x)."""
    return _load().oracle_besselk_scaled(float(nu), float(x))


def dbesselk_dnu(nu: float, x: float) -> float:
    """dK_nu(x)/dnu (the DLMF 10.32.9 integral differentiated in nu)."""
    return _load().oracle_dbesselk_dnu(float(nu), float(x))


def digamma(x: float) -> float:
    return _load().oracle_digamma(float(x))


def matern(theta, r: float) -> float:
    """Eq. 3 at distance r (log-space evaluation)."""
    th = _f64(theta)
    return _load().oracle_matern(_p(th), float(r))


def matern_direct(theta, r: float) -> float:
    """Eq. 3 at distance r, evaluated term by term as printed."""
    th = _f64(theta)
    return _load().oracle_matern_direct(_p(th), float(r))


def matern_grad(theta, r: float) -> np.ndarray:
    """(dSigma/dsigma^2, dSigma/dbeta, dSigma/dnu) at distance r."""
    th = _f64(theta)
    out = np.zeros(3)
    _load().oracle_matern_grad(_p(th), float(r), _p(out))
    return out


def covariance(locs, theta) -> np.ndarray:
    """Full n x n Matérn covariance (Eq. 3) for n x 2 locations."""
    locs = _f64(locs).reshape(-1, 2)
    n = locs.shape[0]
    th = _f64(theta)
    S = np.empty((n, n))
    _load().oracle_covariance(n, _p(locs), _p(th), _p(S))
    return S


def covariance_entries(locs, theta, rows, cols) -> np.ndarray:
    """Sigma[rows[k], cols[k]] for sampled checks at large n."""
    locs = _f64(locs).reshape(-1, 2)
    th = _f64(theta)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(rows.shape[0])
    _load().oracle_covariance_entries(rows.shape[0], rows.ctypes.data_as(_PI64), cols.ctypes.data_as(_PI64),
                                      _p(locs), _p(th), _p(out))
    return out


def cholesky(A) -> tuple[np.ndarray, int]:
    """Unblocked lower Cholesky; returns (L with zero upper part, info)."""
    L = _f64(A).copy()
    n = L.shape[0]
    info = int(_load().oracle_cholesky(n, _p(L)))
    return np.tril(L), info


def loglik(locs, Z, theta) -> dict:
    """Eq. 2 log-likelihood (mu = 0).  Returns dict(l, logdet, quad, info)."""
    locs = _f64(locs).reshape(-1, 2)
    Z = _f64(Z)
    th = _f64(theta)
    out = np.zeros(3)
    info = int(_load().oracle_loglik(locs.shape[0], _p(locs), _p(Z), _p(th), _p(out)))
    return {"l": out[0], "logdet": out[1], "quad": out[2], "info": info}


def loglik_grad(locs, Z, theta) -> dict:
    """Log-likelihood plus dl/d(sigma^2, beta, nu)."""
    locs = _f64(locs).reshape(-1, 2)
    Z = _f64(Z)
    th = _f64(theta)
    out = np.zeros(3)
    g = np.zeros(3)
    info = int(_load().oracle_loglik_grad(locs.shape[0], _p(locs), _p(Z), _p(th), _p(out), _p(g)))
    return {"l": out[0], "logdet": out[1], "quad": out[2], "grad": g, "info": info}


def simulate(locs, theta, eps) -> np.ndarray:
    """Z = L eps with L L^T = Sigma(theta) (exact synthetic realisation)."""
    locs = _f64(locs).reshape(-1, 2)
    th = _f64(theta)
    eps = _f64(eps)
    Z = np.empty(locs.shape[0])
    info = int(_load().oracle_simulate(locs.shape[0], _p(locs), _p(th), _p(eps), _p(Z)))
    if info != 0:
        raise ValueError("Sigma(theta) is not positive definite (pivot %d)" % (info - 1))
    return Z


def predict(locs, Z, theta, new_locs) -> tuple[np.ndarray, np.ndarray]:
    """Kriging at new locations: (mean, variance), zero mean (Section IV's exact_predict)."""
    locs = _f64(locs).reshape(-1, 2)
    new_locs = _f64(new_locs).reshape(-1, 2)
    Z = _f64(Z)
    th = _f64(theta)
    m = new_locs.shape[0]
    mean = np.empty(m)
    var = np.empty(m)
    info = int(_load().oracle_predict(locs.shape[0], _p(locs), _p(Z), _p(th), m, _p(new_locs), _p(mean), _p(var)))
    if info != 0:
        raise ValueError("Sigma(theta) is not positive definite (pivot %d)" % (info - 1))
    return mean, var


def fisher(locs, theta) -> np.ndarray:
    """Fisher information I_kl = 1/2 tr(Sigma^-1 D_k Sigma^-1 D_l), 3 x 3 (exact_fisher)."""
    locs = _f64(locs).reshape(-1, 2)
    th = _f64(theta)
    out = np.empty(9)
    info = int(_load().oracle_fisher(locs.shape[0], _p(locs), _p(th), _p(out)))
    if info != 0:
        raise ValueError("Sigma(theta) is not positive definite (pivot %d)" % (info - 1))
    return out.reshape(3, 3)


def set_model(nugget: float = 0.0, metric: int = 0, radius: float = 6371.0) -> None:
    """Model options for every later call: nugget tau^2 on the diagonal; metric 0 Euclidean,
    1 great circle between (longitude, latitude) in degrees on a sphere of this radius."""
    _load().oracle_set_model(float(nugget), int(metric), float(radius))
