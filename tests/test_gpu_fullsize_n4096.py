"""Full-size kernel geometries of the precision and learned workloads against
the oracle, in the launch configuration bench.py times.

  * precision workload: n = m = 4096 (d = 4096, 2049 bases), 4096 queries
    x = A^T z with z 32-sparse +-1/sqrt(32), eps = 0.09, J = 1000, K = 2,
    S = 320; bfloat16 representation (68.75 GB: the tensor-core preprocess and
    query_kernel<bfloat16, 2 granules, x in shared memory>) and float32
    (137.5 GB: the cluster preprocess and query_kernel<float, 4, x in shared
    memory>);
  * learned-form plan: n = m = 2048 padded to d = 4096 (68.75 GB float32,
    query_kernel<float, 2, x in shared memory>), z 32-sparse in 4 runs of 8.

Sampled queries are checked element by element against the oracle's
streaming step (rows A s_l computed lazily): the drawn indices bit for bit,
the coefficients, mu within the stated bounds, the thresholded output
exactly.  Every query is checked against the dense truth h_eps(Ax) (a
property that holds at any size)."""
import numpy as np
import pytest

from gpu_common import build_and_load, f32, okd, oq, oracle_mu_bound_bf16, torch_cuda
import workloads

pytestmark = pytest.mark.gpu


def _dense_support_check(A64, X64, idx, cnt, val, eps):
    """Every query: the output is h_eps(Ax) (indices exactly, values 1e-5)."""
    V = X64 @ A64.T
    misses = 0
    for q in range(X64.shape[0]):
        truth = np.nonzero(np.abs(V[q]) >= eps)[0]
        got = idx[q, :cnt[q]]
        if not np.array_equal(got, truth):
            misses += 1
            continue
        np.testing.assert_allclose(val[q, :cnt[q]], V[q, truth], rtol=0, atol=1e-5)
    return misses


def _oracle_check(A64, X64, res, wl, k, q, dtype, tc_stages):
    idx, val, cnt, mu, ells, coef = res
    m, n = A64.shape
    d = 1 << k
    L = d * (d // 2 + 1)
    N = wl.J * wl.K
    ell_ref = oq.sample_indices(wl.seed_apply, q, N, L)
    np.testing.assert_array_equal(ells[q], ell_ref)                       # a3
    s_rows = np.stack([okd.sample_vector(l, n, k) for l in ell_ref])
    x = X64[q]
    c_ref = s_rows @ x
    np.testing.assert_allclose(coef[q], c_ref, rtol=0, atol=2e-6 * np.abs(x).sum() + 1e-7)  # a4
    rows = s_rows @ A64.T                                                 # (N, m) = A s_l
    mu_ref = oq.median_of_means(rows * c_ref[:, None], wl.J, wl.K)       # a5, a6
    if dtype == "f32":
        tol = 1e-4 * np.abs(mu_ref).max()
        np.testing.assert_allclose(mu[q], mu_ref, rtol=0, atol=tol)
    else:
        norms = np.linalg.norm(A64, axis=1) if tc_stages else None
        tol_vec = (oracle_mu_bound_bf16(rows, c_ref, wl.J, wl.K, norms, k) +
                   1e-5 * np.abs(mu_ref).max())
        assert (np.abs(mu[q] - mu_ref) <= tol_vec).all()
        tol = tol_vec.max()
    ref_idx, ref_val = oq.apply_one(A64, None, x, wl.eps, wl.seed_apply, q, wl.J, wl.K, wl.S, k,
                                    lazy=True)                            # a7, a8
    np.testing.assert_array_equal(idx[q, :cnt[q]], ref_idx)
    np.testing.assert_allclose(val[q, :cnt[q]], ref_val, rtol=0, atol=1e-5)
    return mu_ref, tol


def _run(K, torch, wl, A, X, dtype, debug_rows):
    plan = K.KerdockPlan(wl.m, wl.n, J=wl.J, K=wl.K, S=wl.S, dtype=dtype)
    plan.preprocess(torch.from_numpy(A).cuda())
    Xt = torch.from_numpy(X).cuda()
    idx, val, cnt = plan.apply(Xt, wl.eps, wl.seed_apply)       # the bench's entry point
    dbg = plan.apply(Xt[debug_rows], wl.eps, wl.seed_apply, debug=True)
    plan.sync()
    out = tuple(t.cpu().numpy() for t in (idx, val, cnt))
    dbg = tuple(t.cpu().numpy() for t in dbg)
    plan.close()
    del plan
    torch.cuda.empty_cache()
    return out, dbg


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_n4096_precision_workload_fullsize(dtype):
    torch = torch_cuda()
    K = build_and_load()
    wl = workloads.WORKLOADS["n4096_bf16"]
    A = wl.make_A().astype(np.float32)
    X = workloads.queries_from_codes(f32(A), wl.make_codes()).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    # the debug launch answers the sampled queries as queries 0..3 of their own
    # launch, so their sampling counters are 0..3: compare with those
    picks = [0, 1, 2047, 4095]
    (idx, val, cnt), dbg = _run(K, torch, wl, A, X, dtype, picks)
    assert _dense_support_check(A64, X64, idx, cnt, val, wl.eps) == 0
    X_picks = X64[picks]
    for q in range(len(picks)):
        _oracle_check(A64, X_picks, dbg, wl, 12, q, dtype, tc_stages=(dtype == "bf16"))


def test_n2048_learned_plan_geometry():
    torch = torch_cuda()
    K = build_and_load()
    wl = workloads.WORKLOADS["n2048_blocks"]
    A = wl.make_A().astype(np.float32)
    X = workloads.queries_from_codes(f32(A), wl.make_codes(q=768)).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    picks = [0, 5, 767]
    (idx, val, cnt), dbg = _run(K, torch, wl, A, X, "f32", picks)
    # every returned value is the exact refinement a_i^T x and passes the
    # threshold; the supports match the dense truth on (nearly) every query
    V = X64 @ A64.T
    for q in range(X.shape[0]):
        got = idx[q, :cnt[q]]
        assert (np.diff(got) > 0).all()
        np.testing.assert_allclose(val[q, :cnt[q]], V[q, got], rtol=0, atol=1e-5)
        assert (np.abs(val[q, :cnt[q]]) >= wl.eps).all()
    # at this J the method itself misses a few entries (support recall 0.9997,
    # 98.9 % of queries exact on the 10k evaluation set): bound both rates
    hit = tot = 0
    for q in range(X.shape[0]):
        truth = np.nonzero(np.abs(V[q]) >= wl.eps)[0]
        hit += len(np.intersect1d(idx[q, :cnt[q]], truth))
        tot += len(truth)
    assert hit / tot >= 0.999
    assert _dense_support_check(A64, X64, idx, cnt, val, wl.eps) <= 0.03 * X.shape[0]
    X_picks = X64[picks]
    for q in range(len(picks)):
        _oracle_check(A64, X_picks, dbg, wl, 12, q, "f32", tc_stages=False)
