"""Shared helpers for the GPU parity tests (imported by tests/test_gpu_*.py)."""
import numpy as np

from oracle import kerdock as okd
from oracle import query as oq


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA (no CPU fallback exists)"
    return torch


def build_and_load():
    from paper_2105_05879_gb300 import build as kbuild
    from paper_2105_05879_gb300 import kerdock as K
    kbuild.build()
    K.load_library()
    return K


def f32(a):
    """The float32 values the GPU sees, promoted back to float64 for the oracle."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def signs_to_bits(words, d):
    """Unpack the device sign table (rows of uint32 words) to a (d/2, d) 0/1 array."""
    rows = words.shape[0]
    bits = np.zeros((rows, d), dtype=np.int64)
    for p in range(d):
        bits[:, p] = (words[:, p // 32] >> np.uint32(p % 32)) & np.uint32(1)
    return bits


def representation_slice(plan, b):
    """(d, m) float64 host copy of basis slice b of the device representation."""
    m = plan.info["m"]
    R = plan.representation()
    return R[b, :, :m].float().cpu().numpy().astype(np.float64)


# Tensor-core preprocessing of a bfloat16 representation (d = 1024 and 4096).
# Besides the final rounding of each entry (2^-8 |R|), the rounding of the
# float16 stage inputs (11 significant bits, rows scaled by powers of two)
# perturbs every entry of R[b][:, i] by a small multiple of its rms over w,
# which is ||a_i|| (W / sqrt(d) is orthogonal): the input, and at d = 1024 the
# 4-point stage's two additions and the first 16-point stage's output, at
# d = 4096 the two intermediate stages, each ~2^-12 ||a_i|| in rms.
TC_ABS = {12: 2.0 ** -8, 10: 2.0 ** -8}


def repr_bound_bf16(R_ref, row_norms=None, k=12):
    """Per-entry bound on |R_bf16 - R_exact|: 2^-8 |R| (final rounding), plus
    TC_ABS[k] * ||a_i|| for the tensor-core stages (row_norms given)."""
    bound = 2.0 ** -8 * np.abs(R_ref)
    if row_norms is not None:
        bound = bound + TC_ABS[k] * np.asarray(row_norms)[None, :]
    return bound


def oracle_mu_bound_bf16(rows, c, J, K, row_norms=None, k=12):
    """Per-entry bound on |mu_bf16 - mu_exact| from the representation bound
    above: |d ybar_k| <= (1/J) sum_j |c_j| bound(R_j), and the median is
    1-Lipschitz in the sup norm, so max_k bounds mu."""
    contrib = np.abs(c)[:, None] * repr_bound_bf16(rows, row_norms, k)
    per_batch = contrib.reshape(K, J, -1).sum(axis=1) / J
    return per_batch.max(axis=0)


def check_topS_valid(sel, mu_ref, S, tol):
    """The selected set is a valid top-S of |mu_ref| up to tol: nothing left out
    is clearly larger than something taken."""
    sel = np.asarray(sel)
    assert len(sel) == S and len(set(sel.tolist())) == S
    assert (np.diff(sel) > 0).all(), "selection must be in ascending index order"
    a = np.abs(mu_ref)
    tau = np.sort(a)[::-1][S - 1]
    mask = np.zeros(len(a), dtype=bool)
    mask[sel] = True
    assert (a[mask] >= tau - tol).all()
    assert (a[~mask] <= tau + tol).all()


def oracle_query(A, R, x, eps, seed, q, J, K, S, k, lazy=False):
    return oq.apply_one(A, R, x, eps, seed, q, J, K, S, k, lazy=lazy, return_mu=True)


__all__ = ["okd", "oq"]
