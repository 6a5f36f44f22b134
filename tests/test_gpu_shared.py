"""The shared-sample batched query (kerdock_apply_shared) against the FP64
oracle: every query of the batch runs Algorithm 1 with the sample indices of
query 0, through the C ABI."""
import math

import numpy as np
import pytest

from gpu_common import build_and_load, check_topS_valid, f32, okd, oq, torch_cuda
from oracle import field as ofield
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    return build_and_load()


def shared_case(K, A, X, J, Kb, S, eps, seed, dtype="f32", flags=0):
    torch = torch_cuda()
    m, n = A.shape
    plan = K.KerdockPlan(m, n, J=J, K=Kb, S=S, dtype=dtype)
    plan.preprocess(torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda())
    Xt = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    out = plan.apply_shared(Xt, eps, seed, flags=flags)
    plan.sync()
    return plan, Xt, tuple(t.cpu().numpy() for t in out)


def oracle_mu(A64, x, seed, J, Kb, k):
    # Algorithm 1's estimate with the samples of query 0
    n = A64.shape[1]
    d = 1 << k
    ells = oq.sample_indices(seed, 0, J * Kb, d * (d // 2 + 1))
    s_rows = np.stack([okd.sample_vector(l, n, k) for l in ells])
    rows = s_rows @ A64.T
    return oq.median_of_means(rows * (s_rows @ x)[:, None], J, Kb)


def test_shared_n64_matches_oracle_with_query0_samples(K):
    wl = workloads.WORKLOADS["n64"]
    A = wl.make_A().astype(np.float32)
    X = workloads.queries_from_codes(f32(A), wl.make_codes()).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    R = okd.representation_lemma6(A64, 6)
    plan, _, (idx, val, cnt) = shared_case(K, A, X, wl.J, wl.K, wl.S, wl.eps, 11)
    for q in range(X.shape[0]):
        ref_idx, ref_val = oq.apply_one(A64, R, X64[q], wl.eps, 11, 0, wl.J, wl.K, wl.S, 6)[:2]
        c = cnt[q]
        np.testing.assert_array_equal(idx[q, :c], ref_idx)
        np.testing.assert_allclose(val[q, :c], ref_val, rtol=0, atol=1e-5)
    plan.close()


@pytest.mark.parametrize("m,n,Kb", [(100, 200, 3), (64, 64, 1), (48, 1000, 4)])
def test_shared_full_output_top_s(K, m, n, Kb):
    # every refined entry returned: the selection is a valid top-S of the
    # oracle's mu for the shared samples, the values are exact a_i^T x
    rng = np.random.default_rng(m + n + Kb)
    A = (rng.standard_normal((m, n)) / math.sqrt(n)).astype(np.float32)
    X = rng.standard_normal((20, n)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    A64, X64 = f32(A), f32(X)
    k = ofield.k_for_dimension(n)
    J, S = 40, 16
    plan, _, (idx, val, cnt) = shared_case(K, A, X, J, Kb, S, 0.1, 5, flags=1)
    for q in range(X.shape[0]):
        mu = oracle_mu(A64, X64[q], 5, J, Kb, k)
        assert cnt[q] == S
        sel = idx[q, :S]
        check_topS_valid(sel, mu, S, 1e-4 * np.abs(mu).max())
        np.testing.assert_allclose(val[q, :S], A64[sel] @ X64[q], rtol=0, atol=1e-5)
    plan.close()


def scores_bound(A64, x, seed, J, Kb, k, dtype):
    # |mu| by the oracle with the shared samples, and a per-entry bound on the
    # scores' error from the arithmetic of the products: coefficients through
    # x = x_hi + x_lo (bfloat16 pieces, 2^-16 relative) against exact +-1 and
    # sqrt(d) entries, float32 accumulation over the 2n columns; batch means
    # through c = c_hi + c_lo (2^-16) against R (float32: R_hi + R_lo, the lo
    # x lo product dropped; bfloat16: R as stored), float32 accumulation over
    # P J columns; and the representation's own error (float32: k butterfly
    # stages, k 2^-23 ||a_i||_1; bfloat16: 2^-8 |R| + 2^-8 ||a_i||).  The
    # median and |.| move no entry by more than the largest batch mean moves.
    m, n = A64.shape
    d = 1 << k
    ells = oq.sample_indices(seed, 0, J * Kb, d * (d // 2 + 1))
    s_rows = np.stack([okd.sample_vector(l, n, k) for l in ells])
    rows = s_rows @ A64.T                       # R[l_j][i]
    c = s_rows @ x
    mu = oq.median_of_means(rows * c[:, None], J, Kb)
    abs_c = np.abs(s_rows) @ np.abs(x)
    u = 2.0 ** -23
    P = 3 if dtype == "f32" else 2
    R = np.abs(rows)
    per = ((2.0 ** -16 + 2 * n * u) * abs_c)[:, None] * R \
        + (3 * 2.0 ** -16 + P * J * u) * np.abs(c)[:, None] * R
    if dtype == "f32":
        per += np.abs(c)[:, None] * (k * u * np.abs(A64).sum(axis=1))[None, :]
    else:
        per += np.abs(c)[:, None] * (2.0 ** -8 * R + 2.0 ** -8 * np.linalg.norm(A64, axis=1)[None, :])
    tol = per.reshape(Kb, J, m).mean(axis=1).max(axis=0)
    return np.abs(mu), tol


@pytest.mark.parametrize("m,n,Kb,J,dtype", [
    (100, 200, 3, 40, "f32"), (64, 64, 1, 40, "f32"), (48, 1000, 4, 40, "f32"),
    (256, 256, 1, 1, "f32"), (1024, 1024, 2, 375, "f32"), (100, 200, 3, 40, "bf16"),
    (1024, 1024, 2, 375, "bf16")])
def test_shared_scores_match_oracle_elementwise(K, m, n, Kb, J, dtype):
    # kerdock_apply_shared_scores: every |mu| entry of every query against the
    # oracle's median of means with the shared samples (query 0's), within
    # twice the worst-case bound of scores_bound; with J = K = 1 each score is
    # one product |c R[l][i]|
    torch = torch_cuda()
    rng = np.random.default_rng(m * 7 + n + Kb)
    A = (rng.standard_normal((m, n)) / math.sqrt(n)).astype(np.float32)
    X = rng.standard_normal((12, n)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    A64, X64 = f32(A), f32(X)
    k = ofield.k_for_dimension(n)
    plan = K.KerdockPlan(m, n, J=J, K=Kb, S=min(16, m), dtype=dtype)
    plan.preprocess(torch.from_numpy(A).cuda())
    Xt = torch.from_numpy(X).cuda()
    got_t = plan.shared_scores(Xt, 7)
    plan.sync()
    got = got_t.cpu().numpy().astype(np.float64)
    worst = 0.0
    for q in range(X.shape[0]):
        ref, tol = scores_bound(A64, X64[q], 7, J, Kb, k, dtype)
        err = np.abs(got[q] - ref)
        assert np.all(err <= 2 * tol + 1e-12), (q, float((err / (tol + 1e-30)).max()))
        worst = max(worst, float((err / (tol + 1e-30)).max()))
    print(f"worst error / bound: {worst:.3f}")
    # the scores are what kerdock_apply_shared ranks: refining them gives its outputs
    ref_t = plan.apply_shared(Xt, 0.05, 7, flags=1)
    plan.sync()
    ref_out = [t.cpu().numpy() for t in ref_t]
    idx, val, cnt = plan.alloc_outputs(X.shape[0])
    scores = torch.from_numpy(got.astype(np.float32)).cuda()
    K.kerdock_refine_scores(plan.handle, Xt.data_ptr(), X.shape[0], Xt.stride(0), scores.data_ptr(),
                            plan.S, 0.05, 1, idx.data_ptr(), val.data_ptr(), cnt.data_ptr())
    plan.sync()
    np.testing.assert_array_equal(cnt.cpu().numpy(), ref_out[2])
    np.testing.assert_array_equal(idx.cpu().numpy(), ref_out[0])
    np.testing.assert_array_equal(val.cpu().numpy(), ref_out[1])
    plan.close()


def test_shared_single_query_equals_apply(K):
    # one query: the shared sample set is that query's own (query 0)
    wl = workloads.WORKLOADS["n1024"]
    A = wl.make_A().astype(np.float32)
    X = workloads.queries_from_codes(f32(A), wl.make_codes(q=1)).astype(np.float32)
    plan, Xt, (idx, val, cnt) = shared_case(K, A, X, wl.J, wl.K, wl.S, wl.eps, 3)
    i2, v2, c2 = (t.cpu().numpy() for t in plan.apply(Xt, wl.eps, 3))
    assert cnt[0] == c2[0]
    np.testing.assert_array_equal(idx[0, :cnt[0]], i2[0, :c2[0]])
    np.testing.assert_allclose(val[0, :cnt[0]], v2[0, :c2[0]], rtol=0, atol=1e-6)
    plan.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_shared_n1024_workload_recovers_dense_truth(K, dtype):
    # the bench workload (1000 queries, J = 375, K = 2) with one shared sample
    # set: every support equals the dense truth
    wl = workloads.WORKLOADS["n1024"]
    A = wl.make_A().astype(np.float32)
    X = workloads.queries_from_codes(f32(A), wl.make_codes()).astype(np.float32)
    plan, _, (idx, val, cnt) = shared_case(K, A, X, wl.J, wl.K, wl.S, wl.eps, wl.seed_apply,
                                           dtype=dtype)
    V = f32(X) @ f32(A).T
    ok = 0
    for q in range(X.shape[0]):
        truth = np.nonzero(np.abs(V[q]) >= wl.eps)[0]
        ok += np.array_equal(idx[q, :cnt[q]], truth)
    assert ok == X.shape[0]
    plan.close()


def test_shared_rejects_small_workspace(K):
    torch = torch_cuda()
    plan = K.KerdockPlan(64, 64, J=8, K=2, S=4)
    plan.preprocess(torch.randn(64, 64, device="cuda"))
    X = torch.randn(3, 64, device="cuda")
    idx, val, cnt = plan.alloc_outputs(3)
    need = K.load_library().kerdock_apply_shared_workspace_bytes(plan.handle, 3)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(K.KerdockError):
        K.kerdock_apply_shared(plan.handle, X.data_ptr(), 3, 64, 0.1, 1, 0, idx.data_ptr(),
                               val.data_ptr(), cnt.data_ptr(), ws.data_ptr(), need - 1)
    plan.close()
