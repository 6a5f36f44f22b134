"""Pins for the oracle's streaming step (Algorithm 1, Lemma 2, Theorem 3).

Checked against: published SplitMix64 vectors (tests/golden), uniformity of the
drawn indices, the exact mean and variance of Lemma 2 by enumerating the whole
design, the failure probability of Theorem 3 at its own J, K, closed-form
medians, and the dense brute-force h_eps(Ax).
"""
import math
import os

import numpy as np
import pytest

from oracle import kerdock, query
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_known_answers():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            seed, vals = line.split(":")
            want = [int(v, 0) for v in vals.split()]
            assert query.splitmix64_stream(int(seed), len(want)) == want


def test_counter_hash_is_the_stream():
    # mix(seed + GAMMA (c+1)) is output c of the sequential generator.
    seed = 987654321
    stream = query.splitmix64_stream(seed, 40)
    for c in range(40):
        assert query.splitmix64_mix((seed + query.GAMMA * (c + 1)) % (1 << 64)) == stream[c]


def test_sample_indices_uniform_and_in_range():
    L = 24                      # d = 4: L = 4 * 3 = 12; use 24 to exercise the multiply
    N = 24000
    ells = query.sample_indices(5, 0, N, L)
    assert ells.min() >= 0 and ells.max() < L
    counts = np.bincount(ells, minlength=L)
    chi2 = ((counts - N / L) ** 2 / (N / L)).sum()
    assert chi2 < 60            # 23 dof: P(chi2 > 60) ~ 4e-5
    # queries draw disjoint counter ranges
    a = query.sample_indices(5, 1, 10, 1 << 40)
    b = query.sample_indices(5, 0, 20, 1 << 40)
    np.testing.assert_array_equal(a, b[10:])


@pytest.mark.parametrize("k,n", [(2, 4), (4, 16), (4, 10), (6, 64)])
def test_lemma2_exact_mean_and_variance(k, n):
    # Enumerate z over the whole design: E[e_i^T y] = (Ax)_i and
    # Var(e_i^T y) = 2 a1^2 (d-1)/(d+2) + a2^2 d/(d+2) with a1 = a_i^T x,
    # a2^2 = |a_i|^2 - a1^2 (proof of Lemma 2), for unit x.
    d = 1 << k
    rng = np.random.default_rng(n)
    m = 7
    A = rng.standard_normal((m, n))
    x = rng.standard_normal(n)
    x /= np.linalg.norm(x)
    S = kerdock.sample_vectors(n, k)
    R = kerdock.representation_lemma6(A, k).reshape(-1, m)
    Y = R * (S @ x)[:, None]                 # rows y_l = (A s_l)(s_l^T x)
    np.testing.assert_allclose(Y.mean(axis=0), A @ x, atol=1e-12)
    a1 = A @ x
    a2sq = (A * A).sum(axis=1) - a1 ** 2
    var = 2 * a1 ** 2 * (d - 1) / (d + 2) + a2sq * d / (d + 2)
    np.testing.assert_allclose(Y.var(axis=0), var, rtol=1e-10)
    assert (Y.var(axis=0) <= 2 * (A * A).sum(axis=1).max() + 1e-12).all()


def test_median_of_means_closed_forms():
    Y = np.arange(12, dtype=float).reshape(12, 1)   # J=3: batch means 1, 4, 7, 10
    assert query.median_of_means(Y, 3, 4)[0] == 5.5  # even K: mean of two middle
    assert query.median_of_means(Y[:9], 3, 3)[0] == 4.0
    assert query.median_of_means(Y, 12, 1)[0] == 5.5
    assert query.median_of_means(Y, 6, 2)[0] == np.mean(Y)  # K = 2 is the mean (Sec. 4)
    rng = np.random.default_rng(1)
    for K in (1, 2, 3, 5, 8):
        Y = rng.standard_normal((K * 4, 9))
        np.testing.assert_allclose(query.median_of_means(Y, 4, K),
                                   np.median(Y.reshape(K, 4, 9).mean(axis=1), axis=0))


def test_top_s_ties_and_order():
    mu = np.array([0.5, -2.0, 2.0, 0.1, -0.5, 2.0])
    assert list(query.top_s(mu, 2)) == [1, 2]
    assert list(query.top_s(mu, 3)) == [1, 2, 5]
    assert list(query.top_s(mu, 4)) == [0, 1, 2, 5]
    assert list(query.top_s(mu, 100)) == list(range(6))


def test_threshold_is_inclusive():
    v = np.array([0.25, -0.25, 0.2499999, -1.0, 0.0])
    np.testing.assert_array_equal(query.hard_threshold(v, 0.25), [0.25, -0.25, 0.0, -1.0, 0.0])
    A = np.eye(5)
    idx, val = query.refine_threshold(A, v, np.array([0, 1, 2, 3, 4]), 0.25)
    assert list(idx) == [0, 1, 3] and list(val) == [0.25, -0.25, -1.0]


def test_theorem3_failure_rate():
    # At J >= 4 e^2 |A|^2 / g^2 and K >= 2 log(m / eta) the event
    # |mu - Ax|_inf >= g has probability <= eta.  d = n = 16, rows unit norm.
    k, n = 4, 16
    A = workloads.random_orthogonal(n, 3)
    gamma, eta = 0.5, 0.2
    J, K = query.theorem3_parameters(1.0, 2 * gamma, 0.0, eta, n)
    S = kerdock.sample_vectors(n, k)
    R = kerdock.representation_lemma6(A, k).reshape(-1, n)
    L = S.shape[0]
    trials, fails = 300, 0
    for t in range(trials):
        x = np.random.default_rng(1000 + t).standard_normal(n)
        x /= np.linalg.norm(x)
        ells = query.sample_indices(77, t, J * K, L)
        Y = R[ells] * (S[ells] @ x)[:, None]
        mu = query.median_of_means(Y, J, K)
        fails += np.abs(mu - A @ x).max() >= gamma
    assert fails / trials <= eta


def test_apply_recovers_dense_truth_small():
    # n = 64 workload: exactly sparse Ax with entries +-1/2 and eps = 1/4.
    wl = workloads.WORKLOADS["n64"]
    A = wl.make_A().astype(np.float32).astype(np.float64)
    X = workloads.queries_from_codes(A, wl.make_codes(q=20)).astype(np.float32).astype(np.float64)
    k = 6
    R = kerdock.representation_lemma6(A, k)
    ok = 0
    for q in range(20):
        idx, val = query.apply_one(A, R, X[q], wl.eps, wl.seed_apply, q, 256, 2, 40, k)
        tidx, tval = query.dense_truth(A, X[q], wl.eps)
        if list(idx) == list(tidx):
            np.testing.assert_allclose(val, tval, atol=1e-12)
            ok += 1
    assert ok == 20


def test_lazy_apply_equals_materialised():
    k, n = 6, 64
    A = workloads.random_orthogonal(n, 9)
    R = kerdock.representation_lemma6(A, k)
    x = workloads.queries_from_codes(A, workloads.sparse_codes(n, 1, 4, 0.5, 4))[0]
    r1 = query.apply_one(A, R, x, 0.25, 3, 5, 32, 3, 40, k, return_mu=True)
    r2 = query.apply_one(A, None, x, 0.25, 3, 5, 32, 3, 40, k, lazy=True, return_mu=True)
    np.testing.assert_array_equal(r1[0], r2[0])
    np.testing.assert_allclose(r1[2], r2[2], atol=1e-12)


def test_theorem3_parameters_hand_values():
    # Theorem 3: J >= 4 e^2 |A|_{2->inf}^2 / gamma^2 and K >= 2 log(m / eta), with
    # gamma = (eps - delta) / 2.  Worked by hand (e^2 = 7.38905...):
    #   a = 1, eps = 0.5, delta = 0:   gamma = 1/4, J = ceil(64 e^2) = ceil(472.90) = 473
    #   m = 1024, eta = 0.01:          K = ceil(2 ln 102400) = ceil(23.07) = 24
    #   a = 2, eps = 1, delta = 0.5:   gamma = 1/4, J = ceil(256 e^2) = ceil(1891.6) = 1892
    #   m = 16, eta = 0.2:             K = ceil(2 ln 80) = ceil(8.76) = 9
    #   m = 1, eta = 1:                K = max(1, ceil(0)) = 1
    #   a = 1/2, eps = 1/2, delta = 0: J = ceil(16 e^2) = ceil(118.2) = 119;
    #   m = 2, eta = 1/2:              K = ceil(2 ln 4) = ceil(2.77) = 3
    # A J from gamma instead of gamma^2 (119 and 473), or from eps instead of
    # gamma (119), or K from log10 (11 and 4), fails one of them.
    assert query.theorem3_parameters(1.0, 0.5, 0.0, 0.01, 1024) == (473, 24)
    assert query.theorem3_parameters(2.0, 1.0, 0.5, 0.2, 16) == (1892, 9)
    assert query.theorem3_parameters(1.0, 0.5, 0.0, 1.0, 1)[1] == 1
    assert query.theorem3_parameters(0.5, 0.5, 0.0, 0.5, 2) == (119, 3)
