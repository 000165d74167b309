"""Host logic of the batched solver's autotune cache (api.autotune_cached), with a stand-in batch:
the first call tunes and stores the per-group choice (tile shape, z-chunks) and the graph length
under a key of GPU name, search space and problem list; later calls with the same key reuse it
through configure(), another GPU, search space or problem list tunes again, and an unreadable
cache file is replaced rather than trusted."""
import json
from types import SimpleNamespace

import pytest
import torch

from paper_1904_03057_gb300 import api


class FakeBatch:
    def __init__(self, result):
        self.result = result
        self.tuned = 0
        self.configured = []

    def autotune(self, reps):
        self.tuned += 1
        return dict(self.result)

    def configure(self, groups, check_every):
        self.configured.append(([(g["degree"], tuple(g["tile"]), g["nzc"]) for g in groups], check_every))


def _res(nzc, check_every, rows=24, ms=1.0):
    return {"check_every": check_every, "ms_per_iteration": ms,
            "groups": [{"degree": 2, "tile": [64, rows], "nzc": nzc, "ms": ms / 2},
                       {"degree": 3, "tile": [64, 16], "nzc": 1, "ms": ms / 2}]}


def _probs(*dims):
    return [SimpleNamespace(nx=a, ny=b, nz=c, degree=n) for a, b, c, n in dims]


@pytest.fixture
def gpu_name(monkeypatch):
    name = {"value": "GPU A"}
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: name["value"])
    return name


def test_tunes_once_then_reuses(tmp_path, gpu_name):
    path = str(tmp_path / "tune.json")
    probs = _probs((48, 64, 80, 2), (96, 96, 96, 3))
    b = FakeBatch(_res(3, 24, rows=32, ms=1.5))
    first = api.autotune_cached(b, probs, path)
    assert first["cached"] is False and b.tuned == 1 and first["groups"][0]["nzc"] == 3
    b2 = FakeBatch(_res(9, 1))
    second = api.autotune_cached(b2, probs, path)
    assert second["cached"] is True and b2.tuned == 0
    assert b2.configured == [([(2, (64, 32), 3), (3, (64, 16), 1)], 24)]
    assert second["groups"][0]["tile"] == [64, 32]
    assert len(json.load(open(path))) == 1


def test_key_includes_gpu_and_problems(tmp_path, gpu_name):
    path = str(tmp_path / "tune.json")
    probs = _probs((48, 64, 80, 2))
    api.autotune_cached(FakeBatch(_res(1, 8)), probs, path)
    gpu_name["value"] = "GPU B"
    b = FakeBatch(_res(2, 16))
    assert api.autotune_cached(b, probs, path)["cached"] is False and b.tuned == 1
    b = FakeBatch(_res(4, 32))
    assert api.autotune_cached(b, _probs((48, 64, 80, 3)), path)["cached"] is False and b.tuned == 1
    assert len(json.load(open(path))) == 3


def test_key_includes_search_space(tmp_path, gpu_name, monkeypatch):
    path = str(tmp_path / "tune.json")
    probs = _probs((48, 64, 80, 2))
    api.autotune_cached(FakeBatch(_res(1, 8)), probs, path)
    monkeypatch.setattr(api, "AUTOTUNE_SPACE", "another search space")
    b = FakeBatch(_res(2, 16))
    assert api.autotune_cached(b, probs, path)["cached"] is False and b.tuned == 1


def test_unreadable_cache_is_replaced(tmp_path, gpu_name):
    path = tmp_path / "tune.json"
    path.write_text("{ not json")
    b = FakeBatch(_res(6, 12))
    res = api.autotune_cached(b, _probs((50, 50, 50, 5)), str(path))
    assert res["cached"] is False and b.tuned == 1
    assert list(json.load(open(path)).values())[0]["groups"][0]["nzc"] == 6
