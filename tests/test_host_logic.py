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


def _schedule_reference(plan_ids, row_bytes, costs, grid):
    # the batch schedule restated: plan groups by first appearance, ordered by
    # decreasing row size (stable); queries by group, then decreasing cost
    # (stable); each onto the least-loaded CTA, lowest index on ties
    import heapq
    first = {}
    for i, p in enumerate(plan_ids):
        first.setdefault(p, (len(first), row_bytes[i]))
    groups = sorted(first, key=lambda p: (-first[p][1], first[p][0]))
    rank = {p: r for r, p in enumerate(groups)}
    qs = sorted(range(len(costs)), key=lambda i: (rank[plan_ids[i]], -costs[i], i))
    heap = [(0.0, c) for c in range(grid)]
    lists = [[] for _ in range(grid)]
    for q in qs:
        load, c = heapq.heappop(heap)
        lists[c].append(q)
        heapq.heappush(heap, (load + costs[q], c))
    return lists


@pytest.mark.parametrize("seed,grid,nplans", [(0, 4, 3), (1, 7, 1), (2, 152, 7), (3, 3, 5)])
def test_batch_schedule_is_plan_major_longest_first(seed, grid, nplans):
    from paper_2105_05879_gb300 import build as kbuild
    from paper_2105_05879_gb300 import kerdock as K
    kbuild.build()
    K.load_library()
    rng = np.random.default_rng(seed)
    count = int(rng.integers(grid, 6 * grid + 20))
    plans = [0x1000 * (p + 1) for p in range(nplans)]
    prow = {p: int(rng.choice([256, 1024, 2048, 4096, 8192, 16384])) for p in plans}
    ids = [plans[int(rng.integers(nplans))] for _ in range(count)]
    rb = [prow[p] for p in ids]
    costs = rng.integers(1, 50, count).astype(np.float64) * 1e6   # repeated values: ties
    got = K.kerdock_debug_batch_schedule(ids, rb, costs, grid)
    assert got == _schedule_reference(ids, rb, costs.tolist(), grid)
    assert sorted(q for lst in got for q in lst) == list(range(count))
    # every CTA runs its queries plan by plan, larger rows first (equal rows:
    # the plan met first in the list), and each plan's longest first
    first = {}
    for i, p in enumerate(ids):
        first.setdefault(p, i)
    for lst in got:
        keys = [(-rb[q], first[ids[q]], -costs[q]) for q in lst]
        assert keys == sorted(keys)
    # greedy balance: no CTA ends more than one query's cost above another
    loads = [sum(costs[q] for q in lst) for lst in got]
    assert max(loads) - min(loads) <= costs.max()


def test_batch_schedule_rejects_bad_arguments():
    from paper_2105_05879_gb300 import build as kbuild
    from paper_2105_05879_gb300 import kerdock as K
    kbuild.build()
    K.load_library()
    for costs in ([1.0, -1.0], [1.0, float("nan")], [float("inf"), 1.0]):
        with pytest.raises(K.KerdockError) as e:
            K.kerdock_debug_batch_schedule([1, 2], [4, 4], costs, 2)
        assert e.value.code == -1
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_debug_batch_schedule([1], [4], [1.0], 0)
    assert e.value.code == -1


def test_clock_sampler_summarises_the_record(tmp_path):
    # nvidia-smi's CSV (no header, no units): the median SM clock under load,
    # the maximum clock, and every throttle reason seen Active; lines that do
    # not parse are skipped
    import bench

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.fh = open(s.path, "w")
    s.fh.write("0, 2070, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
               "0, [N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
               "garbage\n"
               "0, 2070, 2070, 900.0, 0x20, Not Active, Active, Not Active, Not Active\n")
    s.proc = _Proc()
    out = s.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0,
                   "reasons": ["hw_thermal_slowdown", "sw_power_cap"], "samples": 3}
    assert not (tmp_path / "clocks.csv").exists()
    assert bench.ClockSampler(0).stop() is None     # never started: no record
