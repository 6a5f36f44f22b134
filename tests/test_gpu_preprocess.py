"""GPU parity of the plan tables (Lemma 6 step (i)) and the preprocessing
(Lemma 6 steps (ii)-(iii) + identity basis) against the FP64 oracle, through
the C ABI."""
import numpy as np
import pytest

from gpu_common import (build_and_load, f32, okd, repr_bound_bf16, representation_slice,
                        signs_to_bits, torch_cuda)
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    return build_and_load()


@pytest.mark.parametrize("n", [4, 16, 64, 256, 1024, 4096])
def test_sign_table_bit_exact(K, n):
    torch = torch_cuda()
    m = 8 if n == 4096 else 4
    plan = K.KerdockPlan(m, n, J=1, K=1, S=1, dtype="bf16" if n == 4096 else "f32")
    words = plan.signs()
    d = plan.info["d"]
    bits = signs_to_bits(words, d)
    if n <= 1024:
        np.testing.assert_array_equal(bits, okd.sign_matrix(plan.info["k"]))
    else:  # d = 4096: every 17th basis
        for b in range(0, d // 2, 17):
            np.testing.assert_array_equal(bits[b], okd.sign_row(b, 12))
    plan.close()
    torch.cuda.synchronize()


CASES = [  # (m, n, dtype)
    (4, 4, "f32"), (16, 16, "f32"), (64, 64, "f32"), (37, 50, "f32"), (5, 3, "f32"),
    (256, 256, "f32"), (100, 200, "f32"), (33, 1000, "f32"), (64, 64, "bf16"),
    (300, 256, "bf16"),
]


@pytest.mark.parametrize("m,n,dtype", CASES)
def test_preprocess_parity(K, m, n, dtype):
    torch = torch_cuda()
    rng = np.random.default_rng(m * 7919 + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    plan = K.KerdockPlan(m, n, J=1, K=1, S=1, dtype=dtype)
    At = torch.from_numpy(A).cuda()
    plan.preprocess(At)
    plan.sync()
    k, d = plan.info["k"], plan.info["d"]
    Rref = okd.representation_lemma6(f32(A), k)
    Rdev = plan.representation()
    ldr = plan.info["ldr"]
    pad = Rdev[:, :, m:ldr].float()
    assert torch.count_nonzero(pad).item() == 0, "padding entries must be zero"
    Rg = Rdev[:, :, :m].float().cpu().numpy().astype(np.float64)
    for b in range(d // 2 + 1):
        scale = np.abs(Rref[b]).max()
        err = np.abs(Rg[b] - Rref[b]).max()
        if dtype == "f32":
            assert err <= 1e-4 * scale, (b, err, scale)
        else:  # bfloat16 storage: 8 significant bits, round-to-nearest error <= 2^-8 |x|
            assert (np.abs(Rg[b] - Rref[b]) <= 2.0 ** -8 * np.abs(Rref[b]) + 1e-6 * scale).all(), b
    plan.close()


def test_preprocess_identity_matrix_exact(K):
    # A = I: the representation rows are the sample vectors s_l (entries +-1,
    # sqrt(d), 0) -- exact in float32.
    torch = torch_cuda()
    for n in (16, 64, 256):
        plan = K.KerdockPlan(n, n, J=1, K=1, S=1)
        plan.preprocess(torch.eye(n, device="cuda"))
        plan.sync()
        R = plan.representation()[:, :, :n].cpu().numpy().reshape(-1, n).astype(np.float64)
        np.testing.assert_array_equal(R, okd.sample_vectors(n, plan.info["k"]))
        plan.close()


def test_preprocess_n1024_sampled_bases(K):
    # Full-size representation of the n = 1024 workload (2.15 GB float32);
    # the oracle checks a spread of basis slices.
    torch = torch_cuda()
    wl = workloads.WORKLOADS["n1024"]
    A = wl.make_A().astype(np.float32)
    plan = K.KerdockPlan(wl.m, wl.n, J=wl.J, K=wl.K, S=wl.S)
    plan.preprocess(torch.from_numpy(A).cuda())
    plan.sync()
    bases = [0, 1, 2, 77, 255, 256, 400, 511, 512]
    Rref = okd.representation_lemma6(f32(A), 10, bases=bases)
    for t, b in enumerate(bases):
        Rg = representation_slice(plan, b)
        assert np.abs(Rg - Rref[t]).max() <= 1e-4 * np.abs(Rref[t]).max(), b
    plan.close()


@pytest.mark.parametrize("m,n,dtype", [(40, 4096, "f32"), (33, 3000, "f32"), (37, 4096, "f32"),
                                     (70, 2048, "bf16"), (37, 4096, "bf16")])
def test_preprocess_d4096_parity(K, m, n, dtype):
    # d = 4096 (k = 12): the tensor-core kernels (float32 as float16 hi + lo
    # pairs, bfloat16 from float16 stages); the oracle checks a spread of
    # bases, including the identity basis d/2 = 2048.
    torch = torch_cuda()
    rng = np.random.default_rng(m * 31 + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    if m == 37:  # rows of very different magnitudes and an all-zero row
        A[0] *= 1e-6
        A[1] *= 3e4
        A[2] = 0.0
        A[5] *= 2.0 ** -30
    plan = K.KerdockPlan(m, n, J=1, K=1, S=1, dtype=dtype)
    assert plan.info["d"] == 4096
    plan.preprocess(torch.from_numpy(A).cuda())
    plan.sync()
    ldr = plan.info["ldr"]
    Rdev = plan.representation()
    bases = [0, 1, 2, 5, 100, 1023, 1024, 1500, 2046, 2047, 2048]
    Rref = okd.representation_lemma6(f32(A), 12, bases=bases)
    worst = 0.0
    for t_, b in enumerate(bases):
        Rg = Rdev[b].float().cpu().numpy().astype(np.float64)
        assert not np.any(Rg[:, m:ldr]), "padding entries must be zero"
        Rg = Rg[:, :m]
        scale = np.abs(Rref[t_]).max()
        if dtype == "f32":
            # per entry within 1e-5 of its row's norm, the scale of the
            # float32 transform's own error (hi + lo keeps 22 bits per stage)
            norms = np.linalg.norm(f32(A), axis=1)
            err = np.abs(Rg - Rref[t_])
            worst = max(worst, float((err / np.maximum(norms, 1e-300)[None, :]).max()))
            assert (err <= 1e-5 * norms[None, :] + 1e-30).all(), b
            assert err.max() <= 1e-4 * scale, b
        else:
            norms = np.linalg.norm(f32(A), axis=1)
            err = np.abs(Rg - Rref[t_])
            worst = max(worst, float(((err - 2.0 ** -8 * np.abs(Rref[t_])) /
                                      np.maximum(norms, 1e-300)[None, :]).max()))
            assert (err <= repr_bound_bf16(Rref[t_], norms, 12) + 1e-6 * scale).all(), b
    if dtype == "bf16":
        print(f"d=4096 bf16 tensor cores m={m} n={n}: worst (err - 2^-8|R|)/||a_i|| = {worst:.3e}")
    else:
        print(f"d=4096 f32 tensor cores m={m} n={n}: worst err/||a_i|| = {worst:.3e}")
    plan.close()


@pytest.mark.parametrize("m,n,scaled", [(1024, 1024, False), (100, 1000, True), (70, 513, False),
                                        (200, 300, True)])
def test_preprocess_d1024_bf16_tensor_cores(K, m, n, scaled):
    # d = 1024 (k = 10), bfloat16: the tensor-core kernel (64-row tiles, float16
    # stages with a power-of-two scale per row).  Ragged m (a partial last
    # tile, padding rows m..ldr), n < d, and -- with `scaled` -- rows of very
    # different magnitudes and an all-zero row.  Every basis for the smaller
    # cases, a spread of bases at m = n = 1024.
    torch = torch_cuda()
    rng = np.random.default_rng(m * 13 + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    if scaled:
        A[0] *= 1e-6
        A[1] *= 3e4
        A[2] = 0.0
        A[3] *= 2.0 ** -30
    plan = K.KerdockPlan(m, n, J=1, K=1, S=1, dtype="bf16")
    assert plan.info["d"] == 1024
    plan.preprocess(torch.from_numpy(A).cuda())
    plan.sync()
    ldr = plan.info["ldr"]
    Rdev = plan.representation()
    bases = [0, 1, 2, 77, 255, 256, 400, 511, 512] if m == 1024 else list(range(513))
    Rref = okd.representation_lemma6(f32(A), 10, bases=bases)
    norms = np.linalg.norm(f32(A), axis=1)
    worst = 0.0
    for t_, b in enumerate(bases):
        Rg = Rdev[b].float().cpu().numpy().astype(np.float64)
        assert not np.any(Rg[:, m:ldr]), "padding entries must be zero"
        Rg = Rg[:, :m]
        err = np.abs(Rg - Rref[t_])
        assert (err <= repr_bound_bf16(Rref[t_], norms, 10)).all(), b
        rel = err - 2.0 ** -8 * np.abs(Rref[t_])
        worst = max(worst, float((rel / np.maximum(norms, 1e-300)[None, :]).max()))
    print(f"d=1024 bf16 tensor cores m={m} n={n}: worst (err - 2^-8|R|)/||a_i|| = {worst:.3e}")
    plan.close()
