"""Host-side logic of the Python package that needs no GPU: the persistent
cache of autotuned ring geometries and the support-recall measure of the
learned form."""
import json

import numpy as np
import pytest

from paper_2105_05879_gb300 import learned, tuning


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tuning.json"
    monkeypatch.setenv("KERDOCK_TUNING_CACHE", str(path))
    monkeypatch.setattr(tuning, "_device_name", lambda: "GPU-X")
    return path


def test_cache_round_trip_and_unreadable_file(cache):
    assert tuning._load() == {}                      # no file yet
    tuning._store({"a": {"ring_kb": 160, "crows": 8}})
    assert json.loads(cache.read_text()) == {"a": {"ring_kb": 160, "crows": 8}}
    assert tuning._load() == {"a": {"ring_kb": 160, "crows": 8}}
    cache.write_text("{not json")
    assert tuning._load() == {}                      # a damaged cache is ignored


class _Plan:
    def __init__(self, n, dtype, m=None, J=375, K=2, S=160):
        self.info = {"m": m or n, "n": n, "dtype": dtype, "J": J, "K": K, "S": S}


def test_plan_key_buckets_the_batch_size(cache):
    p = _Plan(1024, 0)
    keys = {q: tuning.plan_key(p, q) for q in (1, 2, 3, 4, 5, 1000, 1024, 1025)}
    assert keys[1].endswith("|q1") and keys[2].endswith("|q2")
    assert keys[3] == keys[4] and keys[4].endswith("|q4")
    assert keys[5].endswith("|q8")
    assert keys[1000] == keys[1024] and keys[1025].endswith("|q2048")
    assert keys[1].startswith("GPU-X|plan|m1024|n1024|t0|J375|K2|S160")


class _Batch:
    def __init__(self, specs, result=(128, 4, 2.5)):
        self.specs = specs
        self.result = result
        self.tuned = 0
        self.set = []

    def tune(self, reps):
        self.tuned += 1
        return self.result

    def set_tuning(self, rk, cr):
        self.set.append((rk, cr))


def test_autotune_batch_times_once_then_reads_the_cache(cache):
    specs = [{"plan": _Plan(256, 1)}, {"plan": _Plan(1024, 0)}, {"plan": _Plan(256, 1)}]
    b1 = _Batch(specs)
    assert tuning.autotune_batch(b1, reps=2) == (128, 4, 2.5)
    assert b1.tuned == 1 and b1.set == []
    key = tuning.batch_key(b1)
    assert key == "GPU-X|batch|3|256:1,1024:0"
    assert tuning._load()[key] == {"ring_kb": 128, "crows": 4, "ms": 2.5}
    b2 = _Batch(specs, result=(64, 1, 9.9))           # same shape: no timing, cached geometry
    assert tuning.autotune_batch(b2) == (128, 4, 2.5)
    assert b2.tuned == 0 and b2.set == [(128, 4)]
    b3 = _Batch(specs, result=(64, 1, 9.9))           # use_cache=False always times
    assert tuning.autotune_batch(b3, use_cache=False) == (64, 1, 9.9)
    assert b3.tuned == 1
    assert tuning._load()[key]["ring_kb"] == 128      # and leaves the cache alone


def test_support_recall_counts_entries_and_exact_queries():
    torch = pytest.importorskip("torch")
    idx = torch.tensor([[1, 5, 9, 0], [2, 3, 0, 0], [7, 0, 0, 0]], dtype=torch.int32)
    cnt = torch.tensor([3, 2, 0], dtype=torch.int32)  # query 2 returned nothing
    truth = [np.array([1, 5, 9]), np.array([2, 4]), np.array([7])]
    recall, exact = learned.support_recall(idx, cnt, truth)
    assert recall == pytest.approx(4 / 6)             # 3 + 1 + 0 of 3 + 2 + 1
    assert exact == pytest.approx(1 / 3)              # only query 0 is exact
