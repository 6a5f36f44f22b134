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


def oracle_mu_bound_bf16(rows, c, J, K):
    """Per-entry bound on |mu_bf16 - mu_exact| from rounding each stored entry
    to bfloat16 (8 significant bits, relative error <= 2^-8):
    |d ybar_k| <= 2^-8 (1/J) sum_j |c_j||R_j|,
    and the median is 1-Lipschitz in the sup norm, so max_k bounds mu."""
    contrib = np.abs(rows) * np.abs(c)[:, None]
    per_batch = contrib.reshape(K, J, -1).sum(axis=1) / J
    return 2.0 ** -8 * per_batch.max(axis=0)


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
