"""GPU parity of the streaming step (Algorithm 1) against the FP64 oracle,
through the C ABI: drawn indices (bit-exact), coefficients, the median-of-means
estimate mu, the top-S set, the refined values and the thresholded output."""
import math

import numpy as np
import pytest

from gpu_common import (TC_ABS, build_and_load, check_topS_valid, f32, okd, oq,
                        oracle_mu_bound_bf16, torch_cuda)
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    return build_and_load()


def run_case(K, A, X, J, Kb, S, eps, seed, dtype="f32", flags=0):
    torch = torch_cuda()
    m, n = A.shape
    plan = K.KerdockPlan(m, n, J=J, K=Kb, S=S, dtype=dtype)
    plan.preprocess(torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda())
    Xt = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    out = plan.apply(Xt, eps, seed, flags=flags, debug=True)
    plan.sync()
    idx, val, cnt, mu, ells, coef = (t.cpu().numpy() for t in out)
    return plan, idx, val, cnt, mu, ells, coef


def check_query(A64, R, X64, plan, res, eps, seed, J, Kb, S, k, dtype="f32", lazy=False,
                queries=None, full=False):
    idx, val, cnt, mu, ells, coef = res
    m, n = A64.shape
    d = 1 << k
    L = d * (d // 2 + 1)
    S = min(S, m)
    for q in (queries if queries is not None else range(X64.shape[0])):
        x = X64[q]
        ell_ref = oq.sample_indices(seed, q, J * Kb, L)
        np.testing.assert_array_equal(ells[q], ell_ref)            # a3: bit-exact
        s_rows = np.stack([okd.sample_vector(l, n, k) for l in ell_ref])
        c_ref = s_rows @ x
        np.testing.assert_allclose(coef[q], c_ref, rtol=0, atol=2e-6 * np.abs(x).sum() + 1e-7)
        rows = s_rows @ A64.T if lazy else R.reshape(L, m)[ell_ref]
        mu_ref = oq.median_of_means(rows * c_ref[:, None], J, Kb)
        if dtype == "f32":
            tol = 1e-4 * max(np.abs(mu_ref).max(), 1e-30)
            np.testing.assert_allclose(mu[q], mu_ref, rtol=0, atol=tol)
        else:
            norms = np.linalg.norm(A64, axis=1) if k in TC_ABS else None  # tensor-core stages
            tol_vec = (oracle_mu_bound_bf16(rows, c_ref, J, Kb, norms, k) +
                       1e-5 * np.abs(mu_ref).max())
            assert (np.abs(mu[q] - mu_ref) <= tol_vec).all()
            tol = tol_vec.max()
        v_ref_all = A64 @ x
        if full:
            # every selected entry is returned: check the set and the values
            c = cnt[q]
            assert c == S
            sel = idx[q, :c]
            check_topS_valid(sel, mu_ref, S, 2 * tol)
            np.testing.assert_allclose(val[q, :c], v_ref_all[sel], rtol=0, atol=1e-5)
        else:
            ref_idx, ref_val, ref_mu = oq.apply_one(A64, R, x, eps, seed, q, J, Kb, S, k,
                                                    lazy=lazy, return_mu=True)[:3]
            c = cnt[q]
            got = idx[q, :c]
            assert (np.diff(got) > 0).all()
            # values are exact refinements a_i^T x of the returned indices
            np.testing.assert_allclose(val[q, :c], v_ref_all[got], rtol=0, atol=1e-5)
            assert (np.abs(val[q, :c]) >= eps).all()
            np.testing.assert_array_equal(got, ref_idx)


def test_query_n64_workload(K):
    wl = workloads.WORKLOADS["n64"]
    A = wl.make_A().astype(np.float32)
    X = workloads.queries_from_codes(f32(A), wl.make_codes()).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    R = okd.representation_lemma6(A64, 6)
    plan, *res = run_case(K, A, X, wl.J, wl.K, wl.S, wl.eps, wl.seed_apply)
    check_query(A64, R, X64, plan, res, wl.eps, wl.seed_apply, wl.J, wl.K, wl.S, 6)
    # against the dense truth h_eps(Ax): exact recovery on every query
    idx, val, cnt = res[0], res[1], res[2]
    for q in range(X.shape[0]):
        tidx, tval = oq.dense_truth(A64, X64[q], wl.eps)
        np.testing.assert_array_equal(idx[q, :cnt[q]], tidx)
    plan.close()


@pytest.mark.parametrize("Kb", [1, 3, 4, 5, 17, 24, 32])
def test_query_median_variants(K, Kb):
    # K = 1 (plain mean), odd K (middle value), even K > 2 (two middle values);
    # K > 16 takes the finalizer's median from memory instead of registers
    # (K = 24 is Theorem 3's K at m = 1024, eta = 0.01)
    n = 64
    A = workloads.random_orthogonal(n, 21).astype(np.float32)
    Z = workloads.sparse_codes(n, 24, 4, 0.5, 22)
    X = workloads.queries_from_codes(f32(A), Z).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    R = okd.representation_lemma6(A64, 6)
    J = 48
    plan, *res = run_case(K, A, X, J, Kb, 40, 0.25, 99)
    check_query(A64, R, X64, plan, res, 0.25, 99, J, Kb, 40, 6)
    plan.close()


def test_query_full_output_and_all_rows(K):
    # S = m selects every row: the full output is A x exactly (ascending).
    n = 16
    A = workloads.random_orthogonal(n, 5).astype(np.float32)
    X = np.random.default_rng(6).standard_normal((9, n)).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    R = okd.representation_lemma6(A64, 4)
    plan, *res = run_case(K, A, X, 8, 2, n, 0.0, 7, flags=1)
    idx, val, cnt = res[0], res[1], res[2]
    for q in range(9):
        assert cnt[q] == n
        np.testing.assert_array_equal(idx[q], np.arange(n))
        np.testing.assert_allclose(val[q], A64 @ X64[q], atol=1e-5)
    check_query(A64, R, X64, plan, res, 0.0, 7, 8, 2, n, 4, full=True)
    plan.close()


def test_query_threshold_inclusive_exact(K):
    # A = I, x with entries exactly 0.5 / 0.25: |v| >= eps keeps the tie.
    torch = torch_cuda()
    n = 16
    A = np.eye(n, dtype=np.float32)
    X = np.zeros((3, n), dtype=np.float32)
    X[0, 3] = 0.5
    X[1, [2, 9]] = [0.25, -0.5]
    X[2, 5] = 0.2499999
    plan, *res = run_case(K, A, X, 64, 2, n, 0.25, 1)
    idx, val, cnt = res[0], res[1], res[2]
    assert list(idx[0, :cnt[0]]) == [3] and val[0, 0] == 0.5
    assert list(idx[1, :cnt[1]]) == [2, 9] and list(val[1, :2]) == [0.25, -0.5]
    assert cnt[2] == 0
    plan.close()


@pytest.mark.parametrize("m,n", [(37, 50), (20, 3), (130, 256)])
def test_query_ragged_and_padded(K, m, n):
    # n not a power of four (padding to d, identity samples with w >= n have
    # coefficient 0 but still count), m not a multiple of 8.
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    A /= np.linalg.norm(A, axis=1, keepdims=True)
    X = rng.standard_normal((7, n)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    A64, X64 = f32(A), f32(X)
    k = 2
    while (1 << k) < n:
        k += 2
    R = okd.representation_lemma6(A64, k)
    S = min(10, m)
    plan, *res = run_case(K, A, X, 40, 2, S, 0.3, 12345, flags=1)
    check_query(A64, R, X64, plan, res, 0.3, 12345, 40, 2, S, k, full=True)
    plan.close()


def test_query_bf16_n256(K):
    n = 256
    A = workloads.random_orthogonal(n, 31).astype(np.float32)
    Z = workloads.sparse_codes(n, 16, 8, 1 / math.sqrt(8), 32)
    X = workloads.queries_from_codes(f32(A), Z).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    R = okd.representation_lemma6(A64, 8)
    plan, *res = run_case(K, A, X, 200, 2, 80, 0.5 / math.sqrt(8), 77, dtype="bf16", flags=1)
    check_query(A64, R, X64, plan, res, 0.5 / math.sqrt(8), 77, 200, 2, 80, 8, dtype="bf16",
                full=True)
    plan.close()


def test_query_zero_queries_is_noop(K):
    torch = torch_cuda()
    plan = K.KerdockPlan(16, 16, J=4, K=2, S=4)
    plan.preprocess(torch.eye(16, device="cuda"))
    X = torch.zeros((0, 16), device="cuda")
    idx, val, cnt = plan.apply(X, 0.1, 0)
    plan.sync()
    assert cnt.numel() == 0
    plan.close()


def test_query_apply_before_preprocess_fails(K):
    torch = torch_cuda()
    plan = K.KerdockPlan(16, 16, J=4, K=2, S=4)
    X = torch.zeros((2, 16), device="cuda")
    with pytest.raises(K.KerdockError) as e:
        plan.apply(X, 0.1, 0)
    assert e.value.code == -4
    plan.close()


def test_query_large_K_uses_workspace(K):
    # 2 * K * m * 4 bytes of batch means exceed the kernel's shared-memory
    # budget, so they live in the caller's workspace (K = 16, m = 1024).
    torch = torch_cuda()
    n = 1024
    A = workloads.random_orthogonal(n, 41).astype(np.float32)
    Z = workloads.sparse_codes(n, 5, 8, 0.35, 42)
    X = workloads.queries_from_codes(f32(A), Z).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    J, Kb, S = 24, 16, 64
    plan = K.KerdockPlan(n, n, J=J, K=Kb, S=S)
    assert K.kerdock_apply_workspace_bytes(plan.handle, X.shape[0]) > 0
    plan.preprocess(torch.from_numpy(A).cuda())
    res = plan.apply(torch.from_numpy(X).cuda(), 0.1, 5, flags=1, debug=True)
    plan.sync()
    res = tuple(t.cpu().numpy() for t in res)
    check_query(A64, None, X64, plan, res, 0.1, 5, J, Kb, S, 10, lazy=True, full=True)
    plan.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_query_d4096(K, dtype):
    # n = 4096 (x from shared memory, four sign words per lane), m = 256 rows
    # with orthonormal rows so that Ax = z for x = A^T z.
    torch = torch_cuda()
    m, n = 256, 4096
    Q, _ = np.linalg.qr(np.random.default_rng(51).standard_normal((n, m)))
    A = Q.T.astype(np.float32)
    Z = workloads.sparse_codes(m, 4, 8, 0.35, 52)
    X = (Z @ f32(A)).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    J, Kb, S = 160, 2, 48
    plan, *res = run_case(K, A, X, J, Kb, S, 0.15, 9, dtype=dtype, flags=1)
    check_query(A64, None, X64, plan, res, 0.15, 9, J, Kb, S, 12, dtype=dtype, lazy=True,
                full=True)
    plan.close()


def test_plan_autotune_keeps_results(K, tmp_path, monkeypatch):
    # the ring geometry chosen by the autotuner changes timing, not results
    from paper_2105_05879_gb300 import tuning
    monkeypatch.setenv("KERDOCK_TUNING_CACHE", str(tmp_path / "tune.json"))
    torch = torch_cuda()
    wl = workloads.WORKLOADS["n64"]
    A = wl.make_A().astype(np.float32)
    X = workloads.queries_from_codes(f32(A), wl.make_codes()).astype(np.float32)
    plan = K.KerdockPlan(wl.m, wl.n, J=wl.J, K=wl.K, S=wl.S)
    plan.preprocess(torch.from_numpy(A).cuda())
    Xt = torch.from_numpy(X).cuda()
    ref = [t.cpu().numpy() for t in plan.apply(Xt, wl.eps, 3)]
    rk, cr, ms = tuning.autotune_plan(plan, Xt, wl.eps, 3, reps=2)
    assert (tmp_path / "tune.json").exists()
    rk2, cr2, _ = tuning.autotune_plan(plan, Xt, wl.eps, 3, reps=2)  # from the cache
    assert (rk2, cr2) == (rk, cr)
    got = [t.cpu().numpy() for t in plan.apply(Xt, wl.eps, 3)]
    np.testing.assert_array_equal(got[2], ref[2])
    for q in range(X.shape[0]):
        np.testing.assert_array_equal(got[0][q, :got[2][q]], ref[0][q, :ref[2][q]])
        np.testing.assert_array_equal(got[1][q, :got[2][q]], ref[1][q, :ref[2][q]])
    plan.close()


def test_device_wait_timeout_is_reported_and_recoverable(K):
    # A bounded device wait that runs out records a timeout; kerdock_sync
    # reports it once, clears it, and the plan keeps working (S = m: every row
    # is refined, so the output is exact whatever the sketch).
    torch = torch_cuda()
    plan = K.KerdockPlan(16, 16, J=4, K=2, S=16)
    plan.preprocess(torch.eye(16, device="cuda"))
    K.kerdock_debug_wait_timeout(plan.handle, 2000)
    with pytest.raises(K.KerdockError) as e:
        plan.sync()
    assert e.value.code == -7
    plan.sync()  # cleared
    X = torch.zeros((2, 16), device="cuda")
    X[0, 3] = 1.0
    idx, val, cnt = plan.apply(X, 0.5, 0)
    plan.sync()
    assert cnt.cpu().tolist() == [1, 0] and idx[0, 0].item() == 3
    plan.close()


def test_query_kernel_waits_run_out_and_recover(K):
    # With the poll limit lowered to one poll the query kernel's own waits run
    # out in the middle of normal operation: every role stops (the finalizer
    # warps together), the CTA waits for the row copies it issued, the launch
    # records a timeout that kerdock_sync reports once, and the next launch
    # with the default limit answers exactly as before.
    torch = torch_cuda()
    n = 256
    A = workloads.random_orthogonal(n, 81).astype(np.float32)
    Z = workloads.sparse_codes(n, 64, 8, 0.35, 82)
    X = torch.from_numpy(workloads.queries_from_codes(f32(A), Z).astype(np.float32)).cuda()
    plan = K.KerdockPlan(n, n, J=120, K=2, S=80)
    plan.preprocess(torch.from_numpy(A).cuda())
    ref = [t.cpu().numpy() for t in plan.apply(X, 0.15, 5)]
    plan.sync()
    K.kerdock_debug_set_poll_limit(plan.handle, 1)
    plan.apply(X, 0.15, 5)
    with pytest.raises(K.KerdockError) as e:
        plan.sync()
    assert e.value.code == -7  # KERDOCK_ERR_DEVICE_TIMEOUT
    plan.sync()  # reported once, then cleared
    K.kerdock_debug_set_poll_limit(plan.handle, 0)
    got = [t.cpu().numpy() for t in plan.apply(X, 0.15, 5)]
    plan.sync()
    np.testing.assert_array_equal(got[2], ref[2])
    for q in range(X.shape[0]):
        np.testing.assert_array_equal(got[0][q, :ref[2][q]], ref[0][q, :ref[2][q]])
        np.testing.assert_array_equal(got[1][q, :ref[2][q]], ref[1][q, :ref[2][q]])
    plan.close()
