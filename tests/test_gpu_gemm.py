"""The library's bfloat16 tensor-core product (kerdock_debug_gemm) against
float64 products of the same bfloat16 values, element by element.

The product serves the learned network's layers and the two products of the
shared-sample query.  Two k-major operands take the tcgen05 kernel (TMA,
tensor-memory accumulator), other 16-byte-row layouts the cp.async kernel,
the rest the element-wise kernel; each case below lands on one of them, with
ragged M, N, K (partial tiles and a partial K block) and with K split into
planes.  Float32 accumulation of K products of bfloat16 values (exact in
float32) errs by at most about K * 2^-24 * sum_k |a_k b_k| in any order, the
bound used (with a factor 2)."""
import numpy as np
import pytest

from gpu_common import build_and_load, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    return build_and_load()


def operand(torch, rows, k, major, pitch, seed):
    """rows x k bfloat16 matrix stored k-major (row pitch `pitch`) or
    rows-major (k rows of pitch `pitch`); returns (storage, s_row, s_k, values)."""
    g = torch.Generator().manual_seed(seed)
    vals = torch.randn(rows, k, generator=g).to(torch.bfloat16)
    if major == "k":
        store = torch.zeros(rows, pitch, dtype=torch.bfloat16)
        store[:, :k] = vals
        return store.cuda(), pitch, 1, vals.double().numpy()
    store = torch.zeros(k, pitch, dtype=torch.bfloat16)
    store[:, :rows] = vals.T
    return store.cuda(), 1, pitch, vals.double().numpy()


def run(K, M, N, Kd, a_major="k", b_major="k", a_pitch=None, b_pitch=None, kc=0, seed=0):
    torch = torch_cuda()
    a_pitch = a_pitch or ((Kd if a_major == "k" else M) + 7) // 8 * 8
    b_pitch = b_pitch or ((Kd if b_major == "k" else N) + 7) // 8 * 8
    A, sAm, sAk, a = operand(torch, M, Kd, a_major, a_pitch, seed)
    B, sBn, sBk, b = operand(torch, N, Kd, b_major, b_pitch, seed + 1)
    planes = -(-Kd // kc) if kc else 1
    ldc = N + 3
    C = torch.full((planes, M, ldc), float("nan"), dtype=torch.float32, device="cuda")
    K.kerdock_debug_gemm(A.data_ptr(), sAm, sAk, B.data_ptr(), sBn, sBk, M, N, Kd, kc,
                         C.data_ptr(), ldc, None)
    torch.cuda.synchronize()
    got = C.cpu().double().numpy()
    ref = a @ b.T
    bound = 2 * Kd * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    if kc:
        for z in range(planes):  # each plane is its own slice of K
            sl = slice(z * kc, min(Kd, (z + 1) * kc))
            rz = a[:, sl] @ b[:, sl].T
            bz = 2 * kc * 2.0 ** -24 * (np.abs(a[:, sl]) @ np.abs(b[:, sl]).T) + 1e-30
            assert np.all(np.abs(got[z, :, :N] - rz) <= bz)
        total = got[:, :, :N].sum(axis=0)
    else:
        total = got[0, :, :N]
    assert np.all(np.abs(total - ref) <= bound + 2 * planes * 2.0 ** -24 * np.abs(ref))
    return got


@pytest.mark.parametrize("M,N,Kd", [(128, 64, 64), (200, 100, 300), (1, 8, 16), (333, 130, 1125)])
def test_tcgen05_kmajor_ragged(K, M, N, Kd):
    run(K, M, N, Kd, "k", "k", seed=M + N + Kd)


def test_tcgen05_split_planes(K):
    # the shared-sample coefficient product's shape: q = 1000, N = 750, K = 2n = 2048, 4 slices
    run(K, 1000, 750, 2048, "k", "k", kc=512, seed=7)


def test_tcgen05_split_partial_last_slice(K):
    run(K, 130, 70, 450, "k", "k", kc=192, seed=9)


@pytest.mark.parametrize("am,bm", [("k", "n"), ("m", "n"), ("m", "k")])
def test_async_kernel_transposed_operands(K, am, bm):
    run(K, 150, 90, 200, am, bm, seed=11)


def test_elementwise_kernel_unaligned_pitch(K):
    # odd row pitches: no 16-byte rows, the element-wise kernel
    run(K, 70, 40, 101, "k", "k", a_pitch=101, b_pitch=103, seed=13)


def test_debug_gemm_rejects_bad_split(K):
    torch = torch_cuda()
    A = torch.zeros(8, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(8, 8, dtype=torch.float32, device="cuda")
    with pytest.raises(K.KerdockError):
        K.kerdock_debug_gemm(A.data_ptr(), 64, 1, A.data_ptr(), 64, 1, 8, 8, 64, 32,
                             C.data_ptr(), 8, None)
