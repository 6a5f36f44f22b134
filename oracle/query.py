"""Streaming step of Algorithm 1 and the dense truth -- oracle.

Test infrastructure only (see ``oracle/__init__``).  float64 numpy + exact
Python integers.

Sampling (the paper only says 'uniformly from [L]'; this reading is shared
with the CUDA library as an interface): sample j of query q is
    z = SplitMix64_mix(seed + GAMMA * (q*N + j + 1))  (mod 2^64),
    l = floor(z * L / 2^64),
with SplitMix64 as published by Steele, Lea and Flood (OOPSLA 2014).
Batch k of the median of means holds samples j in [kJ, (k+1)J).
"""
import math

import numpy as np

from . import kerdock

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64_mix(z):
    """The SplitMix64 output function applied to a 64-bit state."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_stream(seed, count):
    """The sequential SplitMix64 generator: state += GAMMA, output mix(state)."""
    state = seed & MASK64
    out = []
    for _ in range(count):
        state = (state + GAMMA) & MASK64
        out.append(splitmix64_mix(state))
    return out


def sample_indices(seed, q, N, L):
    """The N indices l_j drawn for query q (Algorithm 1, 'Draw N := JK
    indices uniformly from [L]'), with replacement."""
    out = np.empty(N, dtype=np.int64)
    base = q * N
    for j in range(N):
        z = splitmix64_mix((seed + GAMMA * (base + j + 1)) & MASK64)
        out[j] = (z * L) >> 64
    return out


def median_of_means(Y, J, K):
    """Theorem 3: ybar_k = (1/J) sum_{j in batch k} y_jk, mu = entrywise median
    over k.  With K even the median is the mean of the two middle values
    (Sec. 4 notes that K = 2 then gives the plain mean).  Y has shape (J*K, m)."""
    Y = np.asarray(Y, dtype=np.float64)
    means = Y.reshape(K, J, -1).mean(axis=1)          # (K, m)
    srt = np.sort(means, axis=0)
    if K % 2 == 1:
        return srt[K // 2]
    return 0.5 * (srt[K // 2 - 1] + srt[K // 2])


def batch_means(Y, J, K):
    Y = np.asarray(Y, dtype=np.float64)
    return Y.reshape(K, J, -1).mean(axis=1)


def top_s(mu, S):
    """Indices of the S entries of largest magnitude (Algorithm 1; Sec. 4 uses
    S = 10s).  Ties go to the smaller index.  Returned in ascending order."""
    mu = np.asarray(mu, dtype=np.float64)
    S = min(S, mu.shape[0])
    order = sorted(range(mu.shape[0]), key=lambda i: (-abs(mu[i]), i))
    return np.array(sorted(order[:S]), dtype=np.int64)


def hard_threshold(v, eps):
    """h_eps(t) = t * 1{|t| >= eps} (Sec. 1.1)."""
    v = np.asarray(v, dtype=np.float64)
    return np.where(np.abs(v) >= eps, v, 0.0)


def refine_threshold(A, x, sel, eps):
    """'Compute A_S x and output the indices and values of entries with
    magnitude at least eps' (Algorithm 1).  Ascending indices."""
    A = np.asarray(A, dtype=np.float64)
    v = A[sel] @ np.asarray(x, dtype=np.float64)
    keep = np.abs(v) >= eps
    return np.asarray(sel)[keep], v[keep]


def coefficients(S_rows, x):
    """c_j = s_{l_j}^T x (Algorithm 1, y_j = (A s_l)(s_l^T x))."""
    return np.asarray(S_rows, dtype=np.float64) @ np.asarray(x, dtype=np.float64)


def apply_one(A, R, x, eps, seed, q, J, K, S, k, lazy=False, return_mu=False):
    """Algorithm 1's streaming step for one query x (global index q).

    R is the (B, d, m) representation, or None with lazy=True, in which case
    the sampled rows A s_l are computed on demand."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    d = 1 << k
    L = d * (d // 2 + 1)
    N = J * K
    ells = sample_indices(seed, q, N, L)
    s_rows = np.stack([kerdock.sample_vector(l, n, k) for l in ells])
    c = coefficients(s_rows, x)
    if lazy:
        rows = s_rows @ A.T                          # (N, m) = (A s_l)^T
    else:
        Rf = np.asarray(R, dtype=np.float64).reshape(L, m)
        rows = Rf[ells]
    Y = rows * c[:, None]
    mu = median_of_means(Y, J, K)
    sel = top_s(mu, S)
    idx, val = refine_threshold(A, x, sel, eps)
    if return_mu:
        return idx, val, mu, ells, c
    return idx, val


def theorem3_parameters(a_row_norm_max, eps, delta, eta, m):
    """J and K of Theorem 3 for the accuracy gamma = (eps - delta)/2 that the
    argument around Algorithm 1 asks of mu, failure probability eta."""
    gamma = (eps - delta) / 2.0
    J = math.ceil(4.0 * math.e ** 2 * a_row_norm_max ** 2 / gamma ** 2)
    K = max(1, math.ceil(2.0 * math.log(m / eta)))
    return J, K


def dense_truth(A, x, eps):
    """Support and values of h_eps(Ax), by the naive dense product."""
    v = hard_threshold(np.asarray(A, dtype=np.float64) @ np.asarray(x, dtype=np.float64), eps)
    idx = np.nonzero(v)[0]
    return idx, v[idx]
