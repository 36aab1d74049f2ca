"""GB300 exact Matérn Gaussian log-likelihood (the ExaGeoStat MLE hot path).

Thin ctypes binding over ``libexa.so`` (declared in ``include/exa.h``): every
function marshals torch device pointers, host scalars and the current CUDA
stream into the C ABI of the same name.  All arithmetic runs in the CUDA
kernels of the library; there is no CPU or PyTorch fallback, and every call
raises if the library is missing or returns an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "EXA_OK", "EXA_ERR_ARG", "EXA_ERR_NOT_SPD", "EXA_ERR_NOMEM", "EXA_ERR_CUDA", "EXA_ERR_TIMEOUT",
    "EXA_ERR_IR_NOCONV", "EXA_FP64", "EXA_MIXED_TF32X3", "EXA_MIXED_BF16X3", "EXA_MIXED_FP32", "ExaError", "Context", "lib",
    "exa_ctx_create", "exa_ctx_destroy", "exa_ctx_set_stream", "exa_last_error", "exa_last_pivot",
    "exa_workspace_bytes", "exa_covariance", "exa_potrf", "exa_loglik", "exa_loglik_ex", "exa_loglik_grad",
    "exa_loglik_batched", "exa_simulate", "ExaResult", "PREC", "exa_gemm_update", "exa_ctx_set_mixed_band", "exa_ctx_set_lookahead", "exa_ctx_set_panel_fusion", "exa_ctx_set_lookahead_late", "exa_ctx_set_refinement", "exa_ctx_set_refinement_quad", "exa_profile_enable",
    "exa_profile_read", "KernelStat", "exa_profile_timeline_enable", "exa_profile_timeline", "TimelineRec", "exa_ctx_set_batched", "exa_ctx_set_batched_mixed", "exa_batched_autotune", "exa_loglik_noalloc", "EXA_GEMM_T3", "EXA_GEMM_OZ", "EXA_GEMM_T3_PAIR", "exa_ctx_set_tc_pairs", "exa_ctx_set_far_tile_margin", "exa_ctx_set_gradient_inverse", "exa_probe_fp64_rate", "exa_predict", "exa_fisher", "exa_ctx_set_model",
    "default_prec", "default_tile",
]

EXA_OK, EXA_ERR_ARG, EXA_ERR_NOT_SPD, EXA_ERR_NOMEM, EXA_ERR_CUDA, EXA_ERR_TIMEOUT, EXA_ERR_IR_NOCONV = range(7)
EXA_FP64, EXA_MIXED_FP32, EXA_MIXED_BF16X3, EXA_MIXED_TF32X3 = 0, 1, 2, 3
EXA_GEMM_T3, EXA_GEMM_OZ, EXA_GEMM_T3_PAIR = 0, 1, 2
PREC = {"fp64": EXA_FP64, "tf32x3": EXA_MIXED_TF32X3, "bf16x3": EXA_MIXED_BF16X3, "fp32": EXA_MIXED_FP32}
_STATUS = {0: "EXA_OK", 1: "EXA_ERR_ARG", 2: "EXA_ERR_NOT_SPD", 3: "EXA_ERR_NOMEM", 4: "EXA_ERR_CUDA",
           5: "EXA_ERR_TIMEOUT", 6: "EXA_ERR_IR_NOCONV"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libexa.so")


class ExaError(RuntimeError):
    def __init__(self, status: int, msg: str, pivot: int = -1):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status
        self.pivot = pivot


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("timed_launches", ctypes.c_int64),
                ("ms", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double),
                ("timed_flops", ctypes.c_double), ("timed_bytes", ctypes.c_double)]


class TimelineRec(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("stream", ctypes.c_int32), ("start_ms", ctypes.c_float),
                ("end_ms", ctypes.c_float)]


class ExaResult(ctypes.Structure):
    _fields_ = [("loglik", ctypes.c_double), ("logdet", ctypes.c_double), ("quad", ctypes.c_double),
                ("ir_resid", ctypes.c_double), ("ir_iters", ctypes.c_int32), ("tile_nb", ctypes.c_int32),
                ("exact_band", ctypes.c_int32), ("n_tiles", ctypes.c_int32), ("ms_gen", ctypes.c_float), ("ms_chol", ctypes.c_float), ("ms_solve", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("quad_err", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)


def lib() -> ctypes.CDLL:
    """The loaded libexa.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libexa.so is not built (%s): run paper_1908_06936_gb300.build.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            sig = {
                "exa_ctx_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, ctypes.c_size_t, ctypes.c_int]),
                "exa_ctx_destroy": (None, [_P]),
                "exa_ctx_set_stream": (ctypes.c_int, [_P, _P]),
                "exa_last_error": (ctypes.c_char_p, [_P]),
                "exa_last_pivot": (_I64, [_P]),
                "exa_workspace_bytes": (ctypes.c_size_t, [_P]),
                "exa_covariance": (ctypes.c_int, [_P, _P, _I64, _PD, _P, _I64]),
                "exa_potrf": (ctypes.c_int, [_P, _P, _I64, _I64]),
                "exa_loglik": (ctypes.c_int, [_P, _P, _P, _PD, _I64, ctypes.c_int, _PD]),
                "exa_loglik_ex": (ctypes.c_int, [_P, _P, _P, _PD, _I64, ctypes.c_int, ctypes.POINTER(ExaResult)]),
                "exa_loglik_grad": (ctypes.c_int, [_P, _P, _P, _PD, _I64, ctypes.c_int, _PD, _PD]),
                "exa_loglik_batched": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_I64), ctypes.POINTER(_P),
                                                      ctypes.POINTER(_P), _P, ctypes.c_int, _P, _P]),
                "exa_simulate": (ctypes.c_int, [_P, _P, _P, _PD, _I64, ctypes.c_int, _P]),
                "exa_ctx_set_mixed_band": (ctypes.c_int, [_P, ctypes.c_int]),
                "exa_ctx_set_lookahead": (ctypes.c_int, [_P, ctypes.c_int]),
                "exa_ctx_set_panel_fusion": (ctypes.c_int, [_P, ctypes.c_int64]),
                "exa_ctx_set_lookahead_late": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int]),
                "exa_ctx_set_refinement": (ctypes.c_int, [_P, ctypes.c_double]),
                "exa_ctx_set_refinement_quad": (ctypes.c_int, [_P, ctypes.c_double]),
                "exa_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
                "exa_loglik_noalloc": (ctypes.c_int, [_P, _P, _P, _PD, _I64, _PD]),
                "exa_ctx_set_batched": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_longlong, ctypes.c_int]),
                "exa_ctx_set_batched_mixed": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
                "exa_ctx_set_tc_pairs": (ctypes.c_int, [_P, ctypes.c_int]),
                "exa_predict": (ctypes.c_int, [_P, _P, _P, _PD, _I64, _P, _I64, _P, _P]),
                "exa_fisher": (ctypes.c_int, [_P, _P, _PD, _I64, _PD]),
                "exa_ctx_set_model": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, ctypes.c_double]),
                "exa_ctx_set_far_tile_margin": (ctypes.c_int, [_P, ctypes.c_int]),
                "exa_ctx_set_gradient_inverse": (ctypes.c_int, [_P, ctypes.c_int]),
                "exa_probe_fp64_rate": (ctypes.c_int, [_P, ctypes.c_int, _PD]),
                "exa_batched_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_I64), ctypes.POINTER(_P),
                                                        ctypes.POINTER(_P), _P, ctypes.c_int, _P, _P,
                                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                        ctypes.POINTER(ctypes.c_float)]),
                "exa_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(KernelStat), ctypes.c_int, ctypes.c_int]),
                "exa_profile_timeline_enable": (ctypes.c_int, [_P, ctypes.c_int]),
                "exa_profile_timeline": (ctypes.c_int, [_P, ctypes.POINTER(TimelineRec), ctypes.c_int, ctypes.c_int]),
                "exa_gemm_update": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _P, _P, _P, _I64,
                                                   ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _theta(theta) -> ctypes.Array:
    t = [float(v) for v in theta]
    if len(t) != 3:
        raise ValueError("theta must have 3 components (sigma^2, beta, nu)")
    return (ctypes.c_double * 3)(*t)


def _dev_ptr(t, name: str, n_expected: int | None = None) -> int:
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64:
        raise TypeError("%s must be float64" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if n_expected is not None and t.numel() != n_expected:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), n_expected))
    return t.data_ptr()


def default_prec() -> int:
    """Precision of a Context evaluation whose caller names none: the environment variable EXA_PREC
    (fp64, tf32x3, bf16x3 or fp32, or the numeric code), else EXA_FP64."""
    v = os.environ.get("EXA_PREC", "").strip().lower()
    if not v:
        return EXA_FP64
    if v in PREC:
        return PREC[v]
    if v.isdigit() and int(v) in PREC.values():
        return int(v)
    raise ValueError("EXA_PREC=%r: expected one of %s or its code" % (v, ", ".join(sorted(PREC))))


def default_tile() -> int:
    """FP64 tile of a new Context whose caller names none: the environment variable EXA_TILE (64 or 128),
    else 0 (the library's default)."""
    v = os.environ.get("EXA_TILE", "").strip()
    if not v:
        return 0
    if v not in ("64", "128"):
        raise ValueError("EXA_TILE=%r: expected 64 or 128" % v)
    return int(v)


def _prec(prec) -> int:
    return default_prec() if prec is None else prec


class Context:
    """Owns an exa_ctx bound to a CUDA stream (default: torch's current stream).  tile_nb=None takes
    EXA_TILE from the environment (else the library default); an evaluation with prec=None takes
    EXA_PREC (else EXA_FP64)."""

    def __init__(self, stream=None, workspace_bytes: int = 0, tile_nb: int | None = None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.handle = exa_ctx_create(stream.cuda_stream, workspace_bytes, default_tile() if tile_nb is None else tile_nb)

    def close(self):
        if getattr(self, "handle", None):
            exa_ctx_destroy(self.handle)
            self.handle = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def check(self, status: int):
        if status != EXA_OK:
            raise ExaError(status, exa_last_error(self.handle), exa_last_pivot(self.handle))

    # convenience wrappers (tensors in, Python values out)
    def covariance(self, locs, theta, out=None):
        import torch

        n = locs.shape[0]
        if out is None:
            out = torch.zeros((n, n), dtype=torch.float64, device=locs.device)
        # the library writes column-major (i + j*ld); a row-major torch (n, n) buffer viewed
        # as column-major is its transpose, so the lower triangle lands in out.T
        self.check(exa_covariance(self.handle, locs, n, theta, out, n))
        return out

    def loglik(self, locs, z, theta, prec=None) -> float:
        return self.loglik_ex(locs, z, theta, prec)["loglik"]

    def loglik_ex(self, locs, z, theta, prec=None) -> dict:
        r = ExaResult()
        st = exa_loglik_ex(self.handle, locs, z, theta, locs.shape[0], _prec(prec), r)
        d = r.as_dict()
        d["status"] = st
        self.check(st)
        return d

    def loglik_grad(self, locs, z, theta, prec=None):
        g = (ctypes.c_double * 3)()
        l = ctypes.c_double()
        self.check(exa_loglik_grad(self.handle, locs, z, theta, locs.shape[0], _prec(prec), l, g))
        return l.value, np.array(g[:])

    def predict(self, locs, z, theta, new_locs, variance=True):
        """Kriging at new locations: (mean, variance or None) as device tensors."""
        import torch

        m = new_locs.shape[0]
        mean = torch.empty(m, dtype=torch.float64, device=new_locs.device)
        var = torch.empty(m, dtype=torch.float64, device=new_locs.device) if variance else None
        self.check(exa_predict(self.handle, locs, z, theta, locs.shape[0], new_locs, m, mean, var))
        return mean, var

    def fisher(self, locs, theta) -> np.ndarray:
        """Fisher information of (sigma^2, beta, nu), 3 x 3."""
        out = (ctypes.c_double * 9)()
        self.check(exa_fisher(self.handle, locs, theta, locs.shape[0], out))
        return np.array(out[:]).reshape(3, 3)

    def simulate(self, locs, eps, theta, prec=None):
        import torch

        z = torch.empty_like(eps)
        self.check(exa_simulate(self.handle, locs, eps, theta, locs.shape[0], _prec(prec), z))
        return z


# --- C-ABI functions, same names --------------------------------------------------

def exa_ctx_create(cuda_stream: int = 0, workspace_bytes: int = 0, tile_nb: int = 0) -> int:
    h = _P()
    st = lib().exa_ctx_create(ctypes.byref(h), _P(cuda_stream or None), int(workspace_bytes), int(tile_nb))
    if st != EXA_OK:
        raise ExaError(st, "exa_ctx_create failed")
    return h.value


def exa_ctx_destroy(ctx: int) -> None:
    lib().exa_ctx_destroy(_P(ctx))


def exa_ctx_set_stream(ctx: int, cuda_stream: int) -> int:
    return lib().exa_ctx_set_stream(_P(ctx), _P(cuda_stream or None))


def exa_ctx_set_mixed_band(ctx: int, band: int) -> int:
    return lib().exa_ctx_set_mixed_band(_P(ctx), int(band))


def exa_ctx_set_lookahead(ctx: int, sms: int) -> int:
    return lib().exa_ctx_set_lookahead(_P(ctx), int(sms))


def exa_ctx_set_refinement(ctx: int, resid_target: float) -> int:
    return lib().exa_ctx_set_refinement(_P(ctx), float(resid_target))


def exa_ctx_set_refinement_quad(ctx: int, tol: float) -> int:
    return lib().exa_ctx_set_refinement_quad(_P(ctx), float(tol))


def exa_ctx_set_lookahead_late(ctx: int, rows: int, sms: int) -> int:
    return lib().exa_ctx_set_lookahead_late(_P(ctx), int(rows), int(sms))


def exa_ctx_set_panel_fusion(ctx: int, min_rows: int) -> int:
    return lib().exa_ctx_set_panel_fusion(_P(ctx), int(min_rows))


def exa_last_error(ctx: int) -> str:
    s = lib().exa_last_error(_P(ctx))
    return s.decode() if s else ""


def exa_last_pivot(ctx: int) -> int:
    return int(lib().exa_last_pivot(_P(ctx)))


def exa_workspace_bytes(ctx: int) -> int:
    return int(lib().exa_workspace_bytes(_P(ctx)))


def exa_covariance(ctx: int, locs, n: int, theta, sigma, ld: int) -> int:
    return lib().exa_covariance(_P(ctx), _P(_dev_ptr(locs, "locs", 2 * n)), n, _theta(theta),
                                _P(_dev_ptr(sigma, "sigma")), ld)


def exa_potrf(ctx: int, a, n: int, ld: int) -> int:
    return lib().exa_potrf(_P(ctx), _P(_dev_ptr(a, "a")), n, ld)


def exa_loglik(ctx: int, locs, z, theta, n: int, prec: int, loglik: ctypes.c_double) -> int:
    return lib().exa_loglik(_P(ctx), _P(_dev_ptr(locs, "locs", 2 * n)), _P(_dev_ptr(z, "z", n)), _theta(theta), n,
                            int(prec), ctypes.byref(loglik))


def exa_loglik_ex(ctx: int, locs, z, theta, n: int, prec: int, out: ExaResult) -> int:
    return lib().exa_loglik_ex(_P(ctx), _P(_dev_ptr(locs, "locs", 2 * n)), _P(_dev_ptr(z, "z", n)), _theta(theta),
                               n, int(prec), ctypes.byref(out))


def exa_loglik_grad(ctx: int, locs, z, theta, n: int, prec: int, loglik: ctypes.c_double, grad) -> int:
    return lib().exa_loglik_grad(_P(ctx), _P(_dev_ptr(locs, "locs", 2 * n)), _P(_dev_ptr(z, "z", n)),
                                 _theta(theta), n, int(prec), ctypes.byref(loglik), grad)


def exa_loglik_batched(ctx: int, nrep: int, ns, locs_list, z_list, theta_dev, prec: int, loglik_dev,
                       status_dev) -> int:
    h_n = (_I64 * nrep)(*[int(v) for v in ns])
    pl = (_P * nrep)(*[_dev_ptr(t, "locs[%d]" % i, 2 * int(ns[i])) for i, t in enumerate(locs_list)])
    pz = (_P * nrep)(*[_dev_ptr(t, "z[%d]" % i, int(ns[i])) for i, t in enumerate(z_list)])
    return lib().exa_loglik_batched(_P(ctx), nrep, h_n, pl, pz, _P(_dev_ptr(theta_dev, "theta", 3 * nrep)),
                                    int(prec), _P(_dev_ptr(loglik_dev, "loglik", nrep)),
                                    _P(status_dev.data_ptr()))


def exa_batched_autotune(ctx: int, nrep: int, ns, locs_list, z_list, theta_dev, prec: int, loglik_dev,
                         status_dev) -> tuple:
    """Native tile autotuner of the batched form; returns (status, tile_nb, ctas_per_sm, best_ms)."""
    h_n = (_I64 * nrep)(*[int(v) for v in ns])
    pl = (_P * nrep)(*[_dev_ptr(t, "locs[%d]" % i, 2 * int(ns[i])) for i, t in enumerate(locs_list)])
    pz = (_P * nrep)(*[_dev_ptr(t, "z[%d]" % i, int(ns[i])) for i, t in enumerate(z_list)])
    nb, cps, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_float(0.0)
    rc = lib().exa_batched_autotune(_P(ctx), nrep, h_n, pl, pz, _P(_dev_ptr(theta_dev, "theta", 3 * nrep)), int(prec),
                                    _P(_dev_ptr(loglik_dev, "loglik", nrep)), _P(status_dev.data_ptr()),
                                    ctypes.byref(nb), ctypes.byref(cps), ctypes.byref(ms))
    return rc, nb.value, cps.value, ms.value


def exa_simulate(ctx: int, locs, eps, theta, n: int, prec: int, z) -> int:
    return lib().exa_simulate(_P(ctx), _P(_dev_ptr(locs, "locs", 2 * n)), _P(_dev_ptr(eps, "eps", n)),
                              _theta(theta), n, int(prec), _P(_dev_ptr(z, "z", n)))


def exa_gemm_update(ctx: int, kind: int, m: int, n: int, k: int, a, b, c, ldc: int, store: int) -> int:
    return lib().exa_gemm_update(_P(ctx), int(kind), m, n, k, _P(_dev_ptr(a, "a", m * k)), _P(_dev_ptr(b, "b", n * k)),
                                 _P(_dev_ptr(c, "c")), ldc, int(store))


def exa_profile_enable(ctx: int, on: int) -> int:
    return lib().exa_profile_enable(_P(ctx), int(on))


def exa_profile_read(ctx: int, reset: int = 0) -> list[dict]:
    buf = (KernelStat * 32)()
    k = lib().exa_profile_read(_P(ctx), buf, 32, int(reset))
    return [{"name": buf[i].name.decode(), "launches": buf[i].launches, "timed_launches": buf[i].timed_launches,
             "ms": buf[i].ms, "flops": buf[i].flops, "bytes": buf[i].bytes, "timed_flops": buf[i].timed_flops,
             "timed_bytes": buf[i].timed_bytes} for i in range(k)]


def exa_profile_timeline_enable(ctx: int, on: int) -> int:
    return lib().exa_profile_timeline_enable(_P(ctx), int(on))


def exa_profile_timeline(ctx: int, max_records: int = 1 << 20, reset: int = 0) -> list[tuple]:
    """Timeline of timed launch groups: (kernel class, stream 0/1, start ms, end ms)."""
    buf = (TimelineRec * max_records)()
    k = lib().exa_profile_timeline(_P(ctx), buf, int(max_records), int(reset))
    return [(buf[i].name.decode(), buf[i].stream, buf[i].start_ms, buf[i].end_ms) for i in range(k)]


def exa_ctx_set_batched(ctx: int, tile_nb: int = 0, ctas_per_sm: int = 0, spin_cycles: int = 0,
                        inject_stall: int = 0) -> int:
    return lib().exa_ctx_set_batched(_P(ctx), int(tile_nb), int(ctas_per_sm), int(spin_cycles), int(inject_stall))


def exa_ctx_set_batched_mixed(ctx: int, band: int = 0, max_iter: int = 0) -> int:
    return lib().exa_ctx_set_batched_mixed(_P(ctx), int(band), int(max_iter))


def exa_ctx_set_tc_pairs(ctx: int, on: int) -> int:
    return lib().exa_ctx_set_tc_pairs(_P(ctx), int(on))


def exa_ctx_set_far_tile_margin(ctx: int, bits: int) -> int:
    return lib().exa_ctx_set_far_tile_margin(_P(ctx), int(bits))


def exa_probe_fp64_rate(cuda_stream: int, kind: int) -> float:
    """FP64 issue-rate probe (kind 0: DFMA, 1: DMMA) in TFLOP/s; raises on failure."""
    v = ctypes.c_double()
    st = lib().exa_probe_fp64_rate(_P(cuda_stream or None), int(kind), ctypes.byref(v))
    if st != EXA_OK:
        raise ExaError(st, "exa_probe_fp64_rate failed")
    return v.value


def exa_ctx_set_gradient_inverse(ctx: int, fp64: int) -> int:
    return lib().exa_ctx_set_gradient_inverse(_P(ctx), int(fp64))


def exa_predict(ctx: int, locs, z, theta, n: int, new_locs, m: int, mean, var=None) -> int:
    return lib().exa_predict(_P(ctx), _P(_dev_ptr(locs, "locs", 2 * n)), _P(_dev_ptr(z, "z", n)), _theta(theta), n,
                             _P(_dev_ptr(new_locs, "new_locs", 2 * m) if m else None),
                             int(m), _P(_dev_ptr(mean, "mean", m) if m else None),
                             _P(_dev_ptr(var, "var", m) if var is not None else None))


def exa_fisher(ctx: int, locs, theta, n: int, out) -> int:
    return lib().exa_fisher(_P(ctx), _P(_dev_ptr(locs, "locs", 2 * n)), _theta(theta), n, out)


def exa_ctx_set_model(ctx: int, nugget: float = 0.0, metric: int = 0, radius: float = 0.0) -> int:
    return lib().exa_ctx_set_model(_P(ctx), float(nugget), int(metric), float(radius))


def exa_loglik_noalloc(cuda_stream: int, locs, z, theta, n: int, loglik: ctypes.c_double) -> int:
    """Allocation-free FP64 log-likelihood (n <= 2048); see include/exa.h."""
    return lib().exa_loglik_noalloc(_P(cuda_stream or None), _P(_dev_ptr(locs, "locs", 2 * n)),
                                    _P(_dev_ptr(z, "z", n)), _theta(theta), n, ctypes.byref(loglik))
