"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

The GPU job shards independent query batches over ranks (weak scaling, no
data-path collective); the only cross-rank steps are the timing barrier and
the max over ranks of the step time.  These tests run that logic as two CPU
processes on the gloo backend.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    # each rank's step time differs; every rank must see the slowest one
    step_ms = 1.0 + 0.5 * rank
    got = bench.max_over_ranks(step_ms, world)
    # shard of the n = 64 workload: its own queries and sample stream
    wl = workloads.WORKLOADS["n64"]
    shard = bench.rank_shard(wl, rank)
    codes = wl.make_codes(offset_seed=shard["codes_offset"])
    dist.barrier()
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), got=got, codes=codes,
             seed_apply=shard["seed_apply"])
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_disjoint_shards(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    # max over ranks: both ranks report the slower rank's time
    assert float(r0["got"]) == pytest.approx(1.5)
    assert float(r1["got"]) == pytest.approx(1.5)
    # the two ranks answer different queries with different sample streams
    assert int(r0["seed_apply"]) != int(r1["seed_apply"])
    assert r0["codes"].shape == r1["codes"].shape
    assert not np.array_equal(r0["codes"], r1["codes"])
    s0 = [tuple(np.nonzero(c)[0]) for c in r0["codes"]]
    s1 = [tuple(np.nonzero(c)[0]) for c in r1["codes"]]
    assert s0 != s1


def test_job_rate_counts_all_ranks():
    import bench
    # 1000 queries per rank in 2 ms on the slowest of 4 ranks
    assert bench.job_rate(4, 1000, 2.0) == pytest.approx(2.0e6)
    assert bench.job_rate(1, 1000, 2.0) == pytest.approx(5.0e5)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    wl = __import__("workloads").WORKLOADS["n1024"]
    # rank 0 keeps the workload's own seeds (the single-GPU bench line)
    sh = bench.rank_shard(wl, 0)
    assert sh["codes_offset"] == 0 and sh["seed_apply"] == wl.seed_apply


def test_fig1_errors_worst_case_over_trials():
    import bench
    Z = np.zeros((3, 8))
    Z[0, [1, 5]] = [0.5, -0.5]
    Z[1, [0, 2]] = [0.5, 0.5]
    Z[2, [3, 4]] = [-0.5, 0.5]
    mu = Z.copy()
    mu[1, 7] = 0.25          # worst mu error 0.25 in trial 1
    idx = np.array([[1, 5, 0], [0, 2, 7], [3, 6, 0]])
    val = np.array([[0.5, -0.5, 0.0], [0.5, 0.5, 0.0], [-0.5, 0.1, 0.0]])
    cnt = np.array([3, 3, 2])  # trial 2 misses index 4 and adds 0.1 at 6
    mu_err, h_err, exact = bench.fig1_errors(mu, idx, val, cnt, Z)
    assert mu_err == pytest.approx(0.25)
    assert h_err == pytest.approx(np.sqrt(0.5 ** 2 + 0.1 ** 2))
    assert exact == pytest.approx(2 / 3)


def test_fig1_summary_compacts_the_grid(monkeypatch):
    # the main line carries the paper's cell (J = 375, K = 2) in full and the
    # exact-trial fraction of every (J, K) cell, rows by K, columns by J
    import bench
    grid = [{"J": J, "K": Kk, "exact_frac": round(J / 1000 + Kk / 100, 4), "us_per_query": 1.0}
            for Kk in (1, 2) for J in (375, 25, 1000)]
    monkeypatch.setattr(bench, "run_fig1", lambda *a: {"value": 1.0, "grid": list(grid)})
    line = bench.run_fig1_summary(None, None, None, None)
    assert "grid" not in line
    assert line["at_J375_K2"] == {"J": 375, "K": 2, "exact_frac": 0.395, "us_per_query": 1.0}
    assert line["exact_frac"] == {"J": [25, 375, 1000], "K=1": [0.035, 0.385, 1.01],
                                  "K=2": [0.045, 0.395, 1.02]}


def test_profiled_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    # committed DRAM counters count only while the profiled kernel's own source
    # files are unchanged, and only for the workload they were taken on
    import json
    import bench
    csrc = tmp_path / "paper_2105_05879_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "query.cu").write_text("kernel v1")
    (csrc / "kerdock_internal.cuh").write_text("header")
    (csrc / "other.cu").write_text("unrelated")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.source_hash(bench.KERNEL_SOURCES["query_kernel"])
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"query_kernel": {"source_hash": h, "workload": "n1024", "dram_bytes_per_launch": 123}}))
    assert bench.profiled_traffic("query_kernel", "n1024") == 123
    assert bench.profiled_traffic("query_kernel", "n64") is None
    assert bench.profiled_traffic("preprocess_d1024_kernel", "n1024") is None
    (csrc / "other.cu").write_text("changed elsewhere")      # not one of the kernel's files
    assert bench.profiled_traffic("query_kernel", "n1024") == 123
    (csrc / "query.cu").write_text("kernel v2")               # the kernel changed
    assert bench.profiled_traffic("query_kernel", "n1024") is None
