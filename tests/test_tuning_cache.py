"""The schedule cache of paper_1308_4605_gb300.tuning on CPU: the first call
for a shape autotunes and writes the cache, later calls apply the cached
schedule without timing, and an unreadable cache file is treated as empty.
The C calls are replaced by fakes (no GPU)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if not os.path.exists(os.path.join(ROOT, "paper_1308_4605_gb300", "libstokes_gb300.so")):
    pytest.skip("library not built", allow_module_level=True)
sys.path.insert(0, ROOT)
from paper_1308_4605_gb300 import tuning  # noqa: E402


class _Solver:
    def __init__(self, dim, n, bc):
        self.dim, self.n, self.bc, self.handle = dim, n, bc, object()


@pytest.fixture
def fakes(monkeypatch):
    calls = {"autotune": [], "set": []}

    def autotune(h, precision):
        calls["autotune"].append(precision)
        return {"coarse_level": 4, "threads": 256 if precision else 128, "pair_level": 4,
                "grid_level": 3, "cluster_level": 2}

    def set_schedule(h, precision, lc, th, pl, gl=None, cl=None):
        calls["set"].append((precision, lc, th, pl, gl, cl))

    monkeypatch.setattr(tuning.S, "stk_autotune", autotune)
    monkeypatch.setattr(tuning.S, "stk_set_schedule", set_schedule)
    monkeypatch.setattr(tuning, "_key", lambda sv, p: f"s4|fake-gpu|{sv.dim}|"
                        f"{'x'.join(map(str, sv.n[:sv.dim]))}|{','.join(map(str, sv.bc))}|{p}")
    return calls


def test_first_call_tunes_then_cache_hits(tmp_path, fakes):
    path = str(tmp_path / "sched.json")
    sv = _Solver(3, (128, 128, 128), (0,) * 6)
    a = tuning.tune(sv, 1, path)
    assert fakes["autotune"] == [1] and fakes["set"] == []
    cache = json.load(open(path))
    assert list(cache.values()) == [a]
    b = tuning.tune(sv, 1, path)
    assert b == a and fakes["autotune"] == [1]
    assert fakes["set"] == [(1, 4, 256, 4, 3, 2)]
    tuning.tune(sv, 0, path)                       # another precision is another entry
    assert fakes["autotune"] == [1, 0] and len(json.load(open(path))) == 2
    tuning.tune(_Solver(3, (64, 64, 64), (0,) * 6), 0, path)   # another grid too
    assert fakes["autotune"] == [1, 0, 0] and len(json.load(open(path))) == 3


def test_unreadable_cache_is_retuned(tmp_path, fakes):
    path = str(tmp_path / "sched.json")
    with open(path, "w") as f:
        f.write("{not json")
    sc = tuning.tune(_Solver(2, (64, 64, 1), (0,) * 4), 0, path)
    assert fakes["autotune"] == [0]
    assert json.load(open(path)) and sc["threads"] == 128


def test_cache_path_from_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("STK_TUNING_CACHE", str(tmp_path / "x.json"))
    assert tuning.cache_path() == str(tmp_path / "x.json")
    monkeypatch.delenv("STK_TUNING_CACHE")
    assert tuning.cache_path().endswith(os.path.join(".cache", "stokes_gb300", "schedules.json"))
