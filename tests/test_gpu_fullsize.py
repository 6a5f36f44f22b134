"""The benchmark workload at full size (n = m = 1024, float32 representation,
1000 queries, J = 375, K = 2, S = 160), in the launch configuration bench.py
times.  Sampled queries are checked one by one against the oracle (rows of
the representation computed lazily); every query is checked against the dense
truth h_eps(Ax)."""
import numpy as np
import pytest

from gpu_common import build_and_load, f32, okd, oq, torch_cuda
import workloads

pytestmark = pytest.mark.gpu


def test_n1024_workload_fullsize():
    torch = torch_cuda()
    K = build_and_load()
    wl = workloads.WORKLOADS["n1024"]
    A = wl.make_A().astype(np.float32)
    X = workloads.queries_from_codes(f32(A), wl.make_codes()).astype(np.float32)
    A64, X64 = f32(A), f32(X)
    plan = K.KerdockPlan(wl.m, wl.n, J=wl.J, K=wl.K, S=wl.S)
    plan.preprocess(torch.from_numpy(A).cuda())
    Xt = torch.from_numpy(X).cuda()
    idx, val, cnt, mu, ells, coef = plan.apply(Xt, wl.eps, wl.seed_apply, debug=True)
    idx2, val2, cnt2 = plan.apply(Xt, wl.eps, wl.seed_apply)   # the non-debug entry point
    plan.sync()
    idx, val, cnt, mu = (t.cpu().numpy() for t in (idx, val, cnt, mu))
    ells = ells.cpu().numpy()
    np.testing.assert_array_equal(cnt2.cpu().numpy(), cnt)
    for q in range(X.shape[0]):
        np.testing.assert_array_equal(idx2.cpu().numpy()[q, :cnt[q]], idx[q, :cnt[q]])
    # every query: the thresholded output equals the dense truth
    misses = 0
    for q in range(X.shape[0]):
        tidx, tval = oq.dense_truth(A64, X64[q], wl.eps)
        got = idx[q, :cnt[q]]
        if not np.array_equal(got, tidx):
            misses += 1
            continue
        np.testing.assert_allclose(val[q, :cnt[q]], tval, atol=1e-5)
    assert misses == 0
    # sampled queries against the oracle's own streaming step
    L = wl.n * (wl.n // 2 + 1)
    for q in (0, 1, 517, 999):
        ell_ref = oq.sample_indices(wl.seed_apply, q, wl.J * wl.K, L)
        np.testing.assert_array_equal(ells[q], ell_ref)
        ref_idx, ref_val, ref_mu, _, _ = oq.apply_one(A64, None, X64[q], wl.eps, wl.seed_apply, q,
                                                      wl.J, wl.K, wl.S, 10, lazy=True,
                                                      return_mu=True)
        np.testing.assert_allclose(mu[q], ref_mu, rtol=0, atol=1e-4 * np.abs(ref_mu).max())
        np.testing.assert_array_equal(idx[q, :cnt[q]], ref_idx)
        np.testing.assert_allclose(val[q, :cnt[q]], ref_val, atol=1e-5)
    plan.close()
