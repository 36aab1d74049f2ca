"""Host logic of the batched autotuner's persistent cache (no GPU: the native tuner is faked)."""
import json

import pytest

import paper_1908_06936_gb300 as exa
from paper_1908_06936_gb300 import tune


class FakeCtx:
    handle = 1234

    def check(self, rc):
        assert rc == 0


@pytest.fixture
def fakes(monkeypatch):
    calls = {"tune": 0, "set": []}

    def fake_tune(handle, nrep, ns, locs, zs, th, prec, out, st):
        calls["tune"] += 1
        return 0, 32, 3, 12.5

    def fake_set(handle, tile, cps, spin, stall):
        calls["set"].append((tile, cps))
        return 0

    import torch

    monkeypatch.setattr(exa, "exa_batched_autotune", fake_tune)
    monkeypatch.setattr(exa, "exa_ctx_set_batched", fake_set)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    return calls


def test_key_ignores_replicate_order_and_tracks_what_selects_the_kernel():
    k1 = tune.workload_key("G", 3, 0, [400, 900, 6400])
    assert k1 == tune.workload_key("G", 3, 0, [6400, 400, 900])
    assert k1 != tune.workload_key("G", 0, 0, [400, 900, 6400])
    assert k1 != tune.workload_key("G", 3, 1, [400, 900, 6400])
    assert k1 != tune.workload_key("G", 3, 0, [400, 900, 6401])
    assert k1 != tune.workload_key("H", 3, 0, [400, 900, 6400])


def test_first_call_tunes_and_stores_then_cache_is_applied(tmp_path, fakes):
    path = str(tmp_path / "sub" / "tiles.json")
    ns = [400, 2500, 900]
    r1 = tune.autotune_batched(FakeCtx(), ns, None, None, None, 3, None, None, cache_path=path)
    assert r1 == {"tile_nb": 32, "ctas_per_sm": 3, "ms": 12.5, "cached": False}
    assert fakes["tune"] == 1 and fakes["set"] == []
    db = json.load(open(path))
    assert list(db.values()) == [{"tile_nb": 32, "ctas_per_sm": 3, "ms": 12.5}]
    r2 = tune.autotune_batched(FakeCtx(), list(reversed(ns)), None, None, None, 3, None, None, cache_path=path)
    assert r2["cached"] and (r2["tile_nb"], r2["ctas_per_sm"]) == (32, 3)
    assert fakes["tune"] == 1 and fakes["set"] == [(32, 3)]


def test_no_cache_path_always_tunes(tmp_path, fakes):
    for _ in range(2):
        tune.autotune_batched(FakeCtx(), [100], None, None, None, 0, None, None, cache_path=None)
    assert fakes["tune"] == 2


def test_corrupt_cache_is_replaced(tmp_path, fakes):
    path = tmp_path / "tiles.json"
    path.write_text("{not json")
    r = tune.autotune_batched(FakeCtx(), [100], None, None, None, 0, None, None, cache_path=str(path))
    assert not r["cached"]
    assert len(json.load(open(path))) == 1
