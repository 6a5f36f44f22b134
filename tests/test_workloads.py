"""The seeded input generators follow the Sec. 4 recipe: A random orthogonal,
codes z with exactly s entries of magnitude amp (random signs; uniform or
block supports), queries x = A^T z so that Ax = z, every draw reproducible
from its seed."""
import math

import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("n", [1, 5, 64, 257])
def test_random_orthogonal_is_orthogonal_and_seeded(n):
    Q = workloads.random_orthogonal(n, 3)
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(Q @ Q.T, np.eye(n), atol=1e-12)
    np.testing.assert_array_equal(Q, workloads.random_orthogonal(n, 3))
    if n > 1:
        assert not np.allclose(Q, workloads.random_orthogonal(n, 4))


def test_random_orthogonal_signs_are_balanced():
    # the signs of R's diagonal are moved into Q, so (Haar measure) the
    # first column's entries are symmetric about zero over many draws
    first = np.array([workloads.random_orthogonal(4, s)[0, 0] for s in range(400)])
    assert abs(np.mean(first > 0) - 0.5) < 0.1


@pytest.mark.parametrize("n,s,amp", [(64, 4, 0.5), (1024, 16, 0.25), (300, 300, 1.0)])
def test_sparse_codes_exact_support_and_magnitude(n, s, amp):
    Z = workloads.sparse_codes(n, 50, s, amp, 9)
    assert Z.shape == (50, n)
    for z in Z:
        nz = np.nonzero(z)[0]
        assert len(nz) == s
        np.testing.assert_array_equal(np.abs(z[nz]), amp)
    signs = np.sign(Z[Z != 0])
    assert 0.3 < np.mean(signs > 0) < 0.7
    np.testing.assert_array_equal(Z, workloads.sparse_codes(n, 50, s, amp, 9))


def test_sparse_codes_noise_on_every_entry():
    Z = workloads.sparse_codes(1024, 200, 16, 0.25, 5, noise=1e-3)
    clean = workloads.sparse_codes(1024, 200, 16, 0.25, 5)
    off = Z[clean == 0]
    assert np.all(off != 0)
    assert abs(off.std() / 1e-3 - 1) < 0.05 and abs(off.mean()) < 1e-4
    on = Z[clean != 0]
    assert np.all(np.abs(np.abs(on) - 0.25) < 6e-3)


@pytest.mark.parametrize("n,nb,bl", [(2048, 4, 8), (40, 4, 8), (32, 4, 8), (100, 1, 1)])
def test_block_supports_are_disjoint_runs(n, nb, bl):
    Z = workloads.sparse_codes(n, 300, nb * bl, 1.0, 11, blocks=(nb, bl))
    starts = []
    for z in Z:
        supp = np.sort(np.nonzero(z)[0])
        assert len(supp) == nb * bl and supp[0] >= 0 and supp[-1] < n
        runs = supp.reshape(nb, bl)            # sorted support in nb runs of bl
        np.testing.assert_array_equal(runs - runs[:, :1], np.tile(np.arange(bl), (nb, 1)))
        starts.append(runs[0, 0])
    if n == 32:                                # no free slot: the runs tile [0, n)
        assert set(starts) == {0}
    elif n >= 100:
        assert min(starts) <= n // 10          # the first run's start spreads out
        assert max(starts) >= (n - nb * bl) // 4


def test_queries_give_ax_equal_z():
    A = workloads.random_orthogonal(128, 1)
    Z = workloads.sparse_codes(128, 10, 6, 0.4, 2)
    X = workloads.queries_from_codes(A, Z)
    np.testing.assert_allclose(X @ A.T, Z, atol=1e-12)   # A x_r = z_r for each row


@pytest.mark.parametrize("name", sorted(workloads.WORKLOADS))
def test_workload_parameters_follow_the_recipe(name):
    wl = workloads.WORKLOADS[name]
    assert wl.S == min(10 * wl.s, wl.m)                    # Sec. 4: S = 10 s
    assert wl.noise < wl.eps < wl.amp                      # support above eps, noise below
    assert len({wl.seed_A, wl.seed_queries, wl.seed_apply}) == 3
    if wl.blocks is not None:
        assert wl.blocks[0] * wl.blocks[1] == wl.s
    if wl.amp != 0.25 and wl.amp != 0.5:
        assert wl.amp == pytest.approx(1 / math.sqrt(wl.s))  # unit-norm codes
