"""Batching form: queries over a mix of plans (sizes, float32 / bfloat16
representations) with per-query sparsity s, J = 24 s, S = 10 s and
eps = 0.5/sqrt(s), answered by one persistent launch replayed from a CUDA
graph.  Each query is checked against the oracle's streaming step (same seed
and sampling counter) and against the dense truth h_eps(Ax)."""
import math

import numpy as np
import pytest

from gpu_common import build_and_load, f32, okd, oq, torch_cuda
import workloads

pytestmark = pytest.mark.gpu


def _setup(K, torch, shapes, counts, rng, s_range=(2, 9)):
    plans, mats, reps = [], [], []
    for (n, dtype), seed in zip(shapes, range(71, 71 + len(shapes))):
        A = workloads.random_orthogonal(n, seed).astype(np.float32)
        plan = K.KerdockPlan(n, n, J=1, K=1, S=1, dtype=dtype)
        plan.preprocess(torch.from_numpy(A).cuda())
        plans.append(plan)
        mats.append(A)
        k = plan.info["k"]
        reps.append(okd.representation_lemma6(f32(A), k) if n <= 256 else None)
    specs, meta = [], []
    for pi, cnt in enumerate(counts):
        n = shapes[pi][0]
        for r in range(cnt):
            s = int(min(rng.integers(*s_range), max(2, n // 8)))
            z = workloads.sparse_codes(n, 1, s, 1 / math.sqrt(s), int(rng.integers(1 << 30)))[0]
            x = (z @ f32(mats[pi])).astype(np.float32)
            Kb = 2 if r % 3 else 3
            J = 24 * s
            spec = dict(plan=plans[pi], x=torch.from_numpy(x).cuda(), J=J, K=Kb, S=min(10 * s, n),
                        eps=0.5 / math.sqrt(s), seed=1000 + pi, index=r)
            specs.append(spec)
            meta.append((pi, x))
    return plans, mats, reps, specs, meta


def _check(batch, specs, meta, mats, reps, shapes, oracle_limit, oracle_dtypes=("f32",)):
    got = batch.results()
    checked_oracle = {}
    for qi, ((pi, x), sp) in enumerate(zip(meta, specs)):
        n, dtype = shapes[pi]
        A64, x64 = f32(mats[pi]), f32(x)
        idx, val = got[qi]
        tidx, tval = oq.dense_truth(A64, x64, sp["eps"])
        np.testing.assert_array_equal(idx, tidx)           # the method recovers h_eps(Ax)
        np.testing.assert_allclose(val, A64[idx] @ x64, atol=1e-5)
        if dtype in oracle_dtypes and checked_oracle.get(pi, 0) < oracle_limit:
            k = batch.specs[qi]["plan"].info["k"]
            ridx, rval = oq.apply_one(A64, reps[pi], x64, sp["eps"], sp["seed"], sp["index"],
                                      sp["J"], sp["K"], sp["S"], k, lazy=reps[pi] is None)
            np.testing.assert_array_equal(idx, ridx)
            np.testing.assert_allclose(val, rval, atol=1e-5)
            checked_oracle[pi] = checked_oracle.get(pi, 0) + 1


def test_batch_mixed_plans_graph_replay():
    torch = torch_cuda()
    K = build_and_load()
    rng = np.random.default_rng(7)
    shapes = [(64, "f32"), (256, "f32"), (256, "bf16"), (1024, "f32"), (16, "bf16")]
    counts = [9, 17, 5, 3, 1]  # uneven per-plan batches
    plans, mats, reps, specs, meta = _setup(K, torch, shapes, counts, rng)
    batch = K.KerdockBatch(specs, graph=True)
    batch.launch()
    batch.sync()
    _check(batch, specs, meta, mats, reps, shapes, oracle_limit=2)
    first = batch.results()
    batch.launch()  # replay: same inputs, same outputs
    batch.sync()
    for a, b in zip(first, batch.results()):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
    # refill the x buffers in place with new queries and replay the graph
    new_meta = []
    for sp, (pi, _) in zip(specs, meta):
        n = shapes[pi][0]
        s = int(round(0.1 * sp["S"]))
        z = workloads.sparse_codes(n, 1, s, 1 / math.sqrt(s), int(rng.integers(1 << 30)))[0]
        x = (z @ f32(mats[pi])).astype(np.float32)
        sp["x"].copy_(torch.from_numpy(x))
        new_meta.append((pi, x))
    batch.launch()
    batch.sync()
    _check(batch, specs, new_meta, mats, reps, shapes, oracle_limit=1)
    # the autotuner changes the ring geometry, never the results
    rk, cr, ms = batch.tune(reps=2)
    assert rk in (64, 96, 128, 160) and cr in (1, 2, 4, 8) and ms > 0
    before = batch.results()
    batch.launch()
    batch.sync()
    for a, b in zip(before, batch.results()):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_allclose(a[1], b[1], atol=0)
    # re-dealing the queries to other CTAs changes the schedule, never the results
    nq = len(specs)
    for costs in (np.arange(nq, dtype=np.float64), rng.random(nq), np.zeros(nq)):
        batch.set_costs(costs)
        batch.launch()
        batch.sync()
        for a, b in zip(before, batch.results()):
            np.testing.assert_array_equal(a[0], b[0])
            np.testing.assert_allclose(a[1], b[1], atol=0)
    for bad in (np.ones(nq - 1), -np.ones(nq), np.full(nq, np.nan), np.full(nq, np.inf)):
        with pytest.raises(K.KerdockError) as e:
            batch.set_costs(bad)
        assert e.value.code == -1
    # explicit schedules: several queries per CTA, fewer CTAs than the launch
    # (the rest run nothing), an empty list in the middle
    assert batch.ctas == min(nq, torch.cuda.get_device_properties(0).multi_processor_count)
    perm = rng.permutation(nq).tolist()
    for lists in ([perm[i::4] for i in range(4)], [perm[:nq // 2], [], perm[nq // 2:]],
                  [list(range(nq))]):
        batch.set_schedule(lists)
        batch.launch()
        batch.sync()
        for a, b in zip(before, batch.results()):
            np.testing.assert_array_equal(a[0], b[0])
            np.testing.assert_allclose(a[1], b[1], atol=0)
    for bad in ([list(range(nq - 1))], [list(range(nq - 1)) + [0]],
                [[i] for i in range(nq)] + [[]] * (batch.ctas + 1 - nq)):
        with pytest.raises(K.KerdockError) as e:  # not a permutation; too many CTAs
            batch.set_schedule(bad)
        assert e.value.code == -1
    batch.close()
    for p in plans:
        p.close()


def test_batch_rejects_bad_queries():
    torch = torch_cuda()
    K = build_and_load()
    plan = K.KerdockPlan(64, 64, J=1, K=1, S=1)
    x = torch.zeros(64, device="cuda")
    spec = dict(plan=plan, x=x, J=8, K=2, S=8, eps=0.1, seed=0, index=0)
    with pytest.raises(K.KerdockError) as e:  # plan not preprocessed
        K.KerdockBatch([spec])
    assert e.value.code == -4
    plan.preprocess(torch.eye(64, device="cuda"))
    with pytest.raises(K.KerdockError) as e:  # S > m
        K.KerdockBatch([dict(spec, S=65)])
    assert e.value.code == -1
    with pytest.raises(K.KerdockError) as e:  # K > 32
        K.KerdockBatch([dict(spec, K=33)])
    assert e.value.code == -2
    plan.close()


def test_batch_n4096_plan_and_large_sparsities():
    # The batching workload's ranges: the precision workload's plan (n = 4096,
    # bfloat16, 68.75 GB: x in shared memory, rows of several granules per
    # gather thread) next to float32 plans, with s ~ U{4..64} (s <= n/8),
    # J = 24 s, S = 10 s, eps = 0.5/sqrt(s).  Every query against the dense
    # truth; some of every plan against the oracle's streaming step (rows of
    # the representation computed lazily for n >= 1024).
    torch = torch_cuda()
    K = build_and_load()
    rng = np.random.default_rng(17)
    shapes = [(4096, "bf16"), (1024, "f32"), (256, "f32"), (1024, "bf16")]
    counts = [21, 13, 6, 4]
    plans, mats, reps, specs, meta = _setup(K, torch, shapes, counts, rng, s_range=(4, 65))
    assert max(sp["S"] // 10 for sp in specs) > 32  # large sparsities are in the batch
    batch = K.KerdockBatch(specs, graph=True)
    batch.launch()
    batch.sync()
    _check(batch, specs, meta, mats, reps, shapes, oracle_limit=1, oracle_dtypes=("f32", "bf16"))
    batch.close()
    for p in plans:
        p.close()
    torch.cuda.empty_cache()


def test_batches_with_different_layouts_coexist():
    # Each batch's graph keeps its own shared-memory layout; the kernel's
    # process-wide shared-memory cap must admit all of them.  The batch with
    # the larger layout (n = 1024, float32 rows and x) is captured first, the
    # smaller one (n = 64) after it, and both are replayed in turn.
    torch = torch_cuda()
    K = build_and_load()
    rng = np.random.default_rng(23)
    big_shapes, small_shapes = [(1024, "f32")], [(64, "f32")]
    pb, mb, rb, sb, metab = _setup(K, torch, big_shapes, [6], rng)
    ps, ms_, rs, ss, metas = _setup(K, torch, small_shapes, [5], rng)
    big = K.KerdockBatch(sb, graph=True)
    small = K.KerdockBatch(ss, graph=True)
    for _ in range(2):
        big.launch()
        small.launch()
        big.sync()
        small.sync()
        _check(big, sb, metab, mb, rb, big_shapes, oracle_limit=0)
        _check(small, ss, metas, ms_, rs, small_shapes, oracle_limit=0)
    big.close()
    small.close()
    for p in pb + ps:
        p.close()
