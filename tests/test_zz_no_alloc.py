"""kerdock_apply_noalloc: the allocation-free form of kerdock_apply.

Callers that cannot allocate device memory (inside stream capture, with a
device-memory budget fixed at start-up, or in a host that owns the allocator)
use this entry point; its scratch is a fixed array inside the library.  These
tests call it through the C ABI and check, on two calls in a row, that it
returns what kerdock_apply returns for the same plan, queries and seed, and
that a call needing more scratch than the array holds is refused.  The file is
named to run after every other test.
"""
import numpy as np
import pytest

from gpu_common import build_and_load, f32, torch_cuda
import workloads

pytestmark = pytest.mark.gpu


def _run_noalloc(K, plan, X, eps, seed, flags):
    idx, val, cnt = plan.alloc_outputs(X.shape[0])
    K.kerdock_apply_noalloc(plan.handle, X.data_ptr(), X.shape[0], X.stride(0), float(eps),
                            int(seed), flags, idx.data_ptr(), val.data_ptr(), cnt.data_ptr())
    plan.sync()
    return idx.cpu().numpy(), val.cpu().numpy(), cnt.cpu().numpy()


@pytest.mark.parametrize("m,n,J,Kb,S,dtype,flags", [
    (1024, 1024, 375, 2, 160, "f32", 0),   # the benchmark workload's plan
    (256, 256, 100, 5, 60, "bf16", 1),     # odd K, bfloat16 rows, full output
    (256, 4096, 120, 2, 48, "f32", 1),     # d = 4096
])
def test_noalloc_matches_apply(m, n, J, Kb, S, dtype, flags):
    torch = torch_cuda()
    K = build_and_load()
    if m == n:
        A = workloads.random_orthogonal(n, 61).astype(np.float32)
    else:
        Q, _ = np.linalg.qr(np.random.default_rng(61).standard_normal((n, m)))
        A = np.ascontiguousarray(Q.T, dtype=np.float32)
    Z = workloads.sparse_codes(m, 300, 8, 0.3, 62)
    X = torch.from_numpy((Z @ f32(A)).astype(np.float32)).cuda()
    plan = K.KerdockPlan(m, n, J=J, K=Kb, S=S, dtype=dtype)
    plan.preprocess(torch.from_numpy(A).cuda())
    eps, seed = 0.15, 2024
    ref = plan.apply(X, eps, seed, flags=flags)
    plan.sync()
    ridx, rval, rcnt = (t.cpu().numpy() for t in ref)
    for _ in range(2):
        idx, val, cnt = _run_noalloc(K, plan, X, eps, seed, flags)
        np.testing.assert_array_equal(cnt, rcnt)
        for q in range(X.shape[0]):
            np.testing.assert_array_equal(idx[q, :cnt[q]], ridx[q, :rcnt[q]])
            np.testing.assert_allclose(val[q, :cnt[q]], rval[q, :rcnt[q]], rtol=0, atol=1e-5)
    plan.close()


def test_noalloc_refuses_beyond_its_scratch():
    # 8 * K * ldr * min(q, SMs) bytes of scratch: K = 16, m = 1024 and 1000
    # queries need about 20 MB > 16 MiB on a 152-SM GPU.
    torch = torch_cuda()
    K = build_and_load()
    n = 1024
    plan = K.KerdockPlan(n, n, J=8, K=16, S=32)
    plan.preprocess(torch.eye(n, device="cuda"))
    X = torch.zeros((1000, n), device="cuda")
    idx, val, cnt = plan.alloc_outputs(1000)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if 8 * 16 * n * min(1000, sms) <= (16 << 20):
        pytest.skip("this GPU has too few SMs to exceed the scratch")
    with pytest.raises(K.KerdockError) as e:
        K.kerdock_apply_noalloc(plan.handle, X.data_ptr(), 1000, n, 0.1, 0, 0, idx.data_ptr(),
                                val.data_ptr(), cnt.data_ptr())
    assert e.value.code == -5  # KERDOCK_ERR_CAPACITY
    plan.close()
