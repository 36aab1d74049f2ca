"""Persistent cache for the batched form's tile autotuner.

The tuning itself is native (``exa_batched_autotune``: every candidate tile and
CTAs-per-SM count is timed with CUDA events on the caller's batch).  This module
keys its choice by GPU name, precision, FP64 band and the multiset of replicate
sizes, stores it in a JSON file, and re-applies it to a context without timing
when the same workload comes back.
"""
from __future__ import annotations

import hashlib
import json
import os

import paper_1908_06936_gb300 as exa

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1908_06936_gb300", "batched_tiles.json")
_FROM_ENV = object()


def default_cache_path() -> str:
    """The cache file when the caller names none: EXA_AUTOTUNE_CACHE from the environment, else DEFAULT_CACHE."""
    return os.environ.get("EXA_AUTOTUNE_CACHE", "").strip() or DEFAULT_CACHE


def workload_key(device_name: str, prec: int, band: int, ns) -> str:
    sizes = ",".join(str(int(v)) for v in sorted(int(v) for v in ns))
    digest = hashlib.sha1(sizes.encode()).hexdigest()[:16]
    return "%s|prec=%d|band=%d|nrep=%d|sizes=%s" % (device_name, int(prec), int(band), len(ns), digest)


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune_batched(ctx, ns, locs_list, z_list, theta_dev, prec: int, loglik_dev, status_dev, band: int = 0,
                     cache_path=_FROM_ENV) -> dict:
    """Pick the batched tile configuration for this workload and apply it to ``ctx``.

    Returns {"tile_nb", "ctas_per_sm", "ms", "cached"}.  ``band`` must match the value
    given to ``exa_ctx_set_batched_mixed`` (it selects the kernel variant).  With
    ``cache_path=None`` nothing is read or written; without it the file is default_cache_path()."""
    import torch

    if cache_path is _FROM_ENV:
        cache_path = default_cache_path()

    key = workload_key(torch.cuda.get_device_name(), prec, band, ns)
    db = _load(cache_path) if cache_path else {}
    if key in db:
        e = db[key]
        ctx.check(exa.exa_ctx_set_batched(ctx.handle, e["tile_nb"], e["ctas_per_sm"], 0, 0))
        return dict(e, cached=True)
    rc, nb, cps, ms = exa.exa_batched_autotune(ctx.handle, len(ns), ns, locs_list, z_list, theta_dev, prec,
                                               loglik_dev, status_dev)
    ctx.check(rc)
    entry = {"tile_nb": nb, "ctas_per_sm": cps, "ms": ms}
    if cache_path:
        db = _load(cache_path)
        db[key] = entry
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dict(entry, cached=False)
