"""Environment defaults of the Python binding (no GPU: the C calls are replaced by recorders).

EXA_PREC sets the precision of a Context evaluation whose caller names none, EXA_TILE the FP64 tile of a new
Context, and EXA_AUTOTUNE_CACHE the batched autotuner's cache file; an explicit argument always wins.
"""
import json

import numpy as np
import pytest
import torch

import paper_1908_06936_gb300 as exa
from paper_1908_06936_gb300 import tune


def test_default_prec(monkeypatch):
    monkeypatch.delenv("EXA_PREC", raising=False)
    assert exa.default_prec() == exa.EXA_FP64
    for v, want in [("tf32x3", exa.EXA_MIXED_TF32X3), ("FP64", exa.EXA_FP64), (" fp32 ", exa.EXA_MIXED_FP32),
                    ("3", exa.EXA_MIXED_TF32X3), ("2", exa.EXA_MIXED_BF16X3)]:
        monkeypatch.setenv("EXA_PREC", v)
        assert exa.default_prec() == want, v
    for bad in ("fp16", "7", "tf32"):
        monkeypatch.setenv("EXA_PREC", bad)
        with pytest.raises(ValueError):
            exa.default_prec()


def test_default_tile(monkeypatch):
    monkeypatch.delenv("EXA_TILE", raising=False)
    assert exa.default_tile() == 0
    monkeypatch.setenv("EXA_TILE", "64")
    assert exa.default_tile() == 64
    for bad in ("96", "x", "256"):
        monkeypatch.setenv("EXA_TILE", bad)
        with pytest.raises(ValueError):
            exa.default_tile()


@pytest.fixture
def recorded(monkeypatch):
    """A Context whose C calls only record their precision and tile arguments."""
    calls = []

    def rec(name, prec_pos):
        def f(*args):
            calls.append((name, args[prec_pos]))
            return exa.EXA_OK
        return f

    monkeypatch.setattr(exa, "exa_loglik_ex", rec("loglik_ex", 5))
    monkeypatch.setattr(exa, "exa_loglik_grad", rec("loglik_grad", 5))
    monkeypatch.setattr(exa, "exa_simulate", rec("simulate", 5))
    monkeypatch.setattr(exa, "exa_ctx_create", lambda stream, ws, tile: calls.append(("create", tile)) or 4242)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: type("S", (), {"cuda_stream": 0})())
    made = []

    def make(**kw):
        c = exa.Context(**kw)
        made.append(c)
        return c

    yield calls, make
    for c in made:
        c.handle = None  # never reaches the real exa_ctx_destroy


def test_context_evaluations_take_the_environment_precision(monkeypatch, recorded):
    calls, make = recorded
    locs, z, th = torch.zeros(4, 2, dtype=torch.float64), torch.zeros(4, dtype=torch.float64), (1.0, 0.1, 0.5)
    c = make()
    monkeypatch.delenv("EXA_PREC", raising=False)
    c.loglik(locs, z, th)
    c.loglik_grad(locs, z, th)
    c.simulate(locs, z, th)
    monkeypatch.setenv("EXA_PREC", "tf32x3")
    c.loglik(locs, z, th)
    c.loglik_ex(locs, z, th)
    c.loglik_grad(locs, z, th)
    c.simulate(locs, z, th)
    c.loglik(locs, z, th, exa.EXA_FP64)  # an explicit precision wins
    assert [p for n, p in calls if n != "create"] == [0, 0, 0, 3, 3, 3, 3, 0]


def test_context_tile_from_the_environment(monkeypatch, recorded):
    calls, make = recorded
    monkeypatch.delenv("EXA_TILE", raising=False)
    make()
    monkeypatch.setenv("EXA_TILE", "64")
    make()
    make(tile_nb=128)  # an explicit tile wins
    assert [t for n, t in calls if n == "create"] == [0, 64, 128]


def test_autotune_cache_file_from_the_environment(monkeypatch, tmp_path):
    path = tmp_path / "tiles.json"
    monkeypatch.setenv("EXA_AUTOTUNE_CACHE", str(path))
    assert tune.default_cache_path() == str(path)
    monkeypatch.setattr(exa, "exa_batched_autotune", lambda *a: (0, 32, 3, 12.5))
    monkeypatch.setattr(exa, "exa_ctx_set_batched", lambda *a: 0)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")

    class FakeCtx:
        handle = 1234

        def check(self, rc):
            assert rc == 0

    got = tune.autotune_batched(FakeCtx(), [400, 900], [None, None], [None, None], None, exa.EXA_MIXED_FP32,
                                None, None)
    assert got["tile_nb"] == 32 and not got["cached"]
    db = json.loads(path.read_text())
    assert list(db) == [tune.workload_key("FakeGPU", exa.EXA_MIXED_FP32, 0, [400, 900])]
    monkeypatch.delenv("EXA_AUTOTUNE_CACHE")
    assert tune.default_cache_path() == tune.DEFAULT_CACHE
