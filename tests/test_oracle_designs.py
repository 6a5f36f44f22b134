"""Pins for the oracle's bases and representation (Prop. 1, 2, 4, Lemma 6).

The MUB vectors are checked against what the paper proves about them
(orthonormality and unbiasedness, Prop. 4; the projective 2-design frame
potentials c_{d,1} = 1/d and c_{d,2} = 3/(d(d+2)), Prop. 1(b)/(c) and Prop. 2;
the inner-product formula in the proof of Prop. 4) and the two routes to the
representation (definition vs. Lemma 6) against each other and against closed
forms (A = I, reconstruction, the frame identity).
"""
import os

import numpy as np
import pytest

from oracle import field, kerdock

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def c_dk(d, k):
    num = np.prod([2 * j + 1 for j in range(k)])
    den = np.prod([d + 2 * j for j in range(k)])
    return num / den


@pytest.mark.parametrize("k", [2, 4, 6])
def test_mubs_orthonormal_and_unbiased(k):
    d = 1 << k
    U = kerdock.mub_vectors(k).reshape(d // 2 + 1, d, d)
    for b in range(d // 2 + 1):
        np.testing.assert_allclose(U[b] @ U[b].T, np.eye(d), atol=1e-12)
        for b2 in range(b + 1, d // 2 + 1):
            G = U[b] @ U[b2].T
            np.testing.assert_allclose(G ** 2, np.full((d, d), 1.0 / d), atol=1e-12)


def test_mubs_k8_sampled_pairs():
    k, d = 8, 256
    U = kerdock.mub_vectors(k).reshape(d // 2 + 1, d, d)
    rng = np.random.default_rng(0)
    for _ in range(24):
        b, b2 = rng.choice(d // 2 + 1, size=2, replace=False)
        np.testing.assert_allclose((U[b] @ U[b2].T) ** 2, 1.0 / d, atol=1e-12)
        np.testing.assert_allclose(U[b] @ U[b].T, np.eye(d), atol=1e-12)


@pytest.mark.parametrize("k", [2, 4, 6])
def test_projective_2_design_frame_potentials(k):
    # Prop. 1(c) for t = 1, 2 and the failure at t = 3 (the union of MUBs is a
    # 2-design, not a 3-design, for d > 2).
    d = 1 << k
    U = kerdock.mub_vectors(k)
    L = U.shape[0]
    assert L == d * (d // 2 + 1)
    G = U @ U.T
    for t in (1, 2):
        assert abs((G ** (2 * t)).sum() / L ** 2 - c_dk(d, t)) < 1e-12
    assert abs((G ** 6).sum() / L ** 2 - c_dk(d, 3)) > 1e-6


@pytest.mark.parametrize("k", [2, 4, 6])
def test_cubature_on_random_vectors(k):
    # Prop. 1(b): (1/L) sum <x,u>^(2t) = c_{d,t} |x|^(2t), t = 1, 2.
    d = 1 << k
    U = kerdock.mub_vectors(k)
    rng = np.random.default_rng(k)
    for _ in range(5):
        x = rng.standard_normal(d)
        ip = U @ x
        for t in (1, 2):
            assert abs(np.mean(ip ** (2 * t)) - c_dk(d, t) * (x @ x) ** t) < 1e-10 * (x @ x) ** t


@pytest.mark.parametrize("k", [2, 4, 6])
def test_tight_frame(k):
    # sum over all bases of B_b^T B_b = (d/2 + 1) I.
    d = 1 << k
    U = kerdock.mub_vectors(k)
    np.testing.assert_allclose(U.T @ U, (d // 2 + 1) * np.eye(d), atol=1e-11)


def test_inner_product_formula_of_prop4_proof():
    # Proof of Prop. 4: |<u_{M,w}, u_{M',w'}>|^2 =
    #   2^-k sum_{p in ker(M+M')} (-1)^(Q_M(p) + Q_M'(p) + (w+w')^T p)
    # for ANY skew-symmetric M, M' (not only Kerdock pairs).
    k = 4
    d = 1 << k
    rng = np.random.default_rng(7)
    P = kerdock.point_bits(k)
    W = kerdock.walsh_matrix(k)

    def basis(M):
        q = np.array([field.quadratic_form(M.tolist(), p) for p in range(d)])
        return W * (1.0 - 2.0 * q)[None, :] / np.sqrt(d)

    for _ in range(10):
        Us = []
        Ms = []
        for _ in range(2):
            T = np.triu(rng.integers(0, 2, size=(k, k)), 1)
            M = T + T.T
            Ms.append(M)
            Us.append(basis(M))
        S = (Ms[0] + Ms[1]) % 2
        ker = [p for p in range(d) if not ((S @ P[p]) % 2).any()]
        for w in range(d):
            for w2 in range(d):
                lhs = (Us[0][w] @ Us[1][w2]) ** 2
                rhs = sum((-1) ** (field.quadratic_form(Ms[0].tolist(), p)
                                   + field.quadratic_form(Ms[1].tolist(), p)
                                   + bin((w ^ w2) & p).count("1")) for p in ker) / d
                assert abs(lhs - rhs) < 1e-12


def test_golden_k2_bases():
    rows = {}
    with open(os.path.join(GOLDEN, "kerdock_n4.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line.startswith("basis"):
                key, val = line.split(":", 1)
                rows[key] = np.array([[float(t) for t in part.split()] for part in val.split("/")])
    S = kerdock.sample_vectors(4, 2).reshape(3, 4, 4)
    for b in range(3):
        np.testing.assert_array_equal(S[b], rows[f"basis{b}"])


@pytest.mark.parametrize("k,m,n", [(2, 3, 4), (2, 5, 3), (4, 16, 16), (4, 7, 11), (6, 64, 64), (6, 20, 50)])
def test_lemma6_equals_definition(k, m, n):
    rng = np.random.default_rng(k * 100 + n)
    A = rng.standard_normal((m, n))
    R1 = kerdock.representation_definition(A, k)
    R2 = kerdock.representation_lemma6(A, k)
    np.testing.assert_allclose(R2, R1, atol=1e-12 * np.abs(R1).max())


@pytest.mark.parametrize("k", [2, 4, 6])
def test_identity_matrix_gives_sample_vectors(k):
    d = 1 << k
    R = kerdock.representation_lemma6(np.eye(d), k)
    np.testing.assert_allclose(R.reshape(-1, d), kerdock.sample_vectors(d, k), atol=1e-12)


@pytest.mark.parametrize("k,n", [(4, 16), (6, 50)])
def test_reconstruction_and_frame_identity(k, n):
    # Per basis: A Pi D_b = T_b W / d with T_b = R[b]^T (W W = d I); and
    # sum_l (A s_l)(A s_l)^T = L A A^T since sum_l s_l s_l^T = L I_n.
    d = 1 << k
    rng = np.random.default_rng(n)
    A = rng.standard_normal((9, n))
    R = kerdock.representation_lemma6(A, k)
    W = kerdock.walsh_matrix(k)
    Apad = np.zeros((9, d))
    Apad[:, :n] = A
    for b in range(d // 2):
        D = 1.0 - 2.0 * kerdock.sign_row(b, k)
        np.testing.assert_allclose(R[b].T @ W / d, Apad * D[None, :], atol=1e-12)
    L = d * (d // 2 + 1)
    Rf = R.reshape(L, -1)
    np.testing.assert_allclose(Rf.T @ Rf, L * A @ A.T, atol=1e-9 * L)


def test_fwht_closed_forms():
    for k in (1, 3, 5):
        d = 1 << k
        np.testing.assert_array_equal(kerdock.fwht_rows(np.eye(d)), kerdock.walsh_matrix(k))
        x = np.random.default_rng(k).standard_normal((3, d))
        np.testing.assert_allclose(kerdock.fwht_rows(kerdock.fwht_rows(x)), d * x, atol=1e-12)


def test_lazy_rows_match_full_representation():
    k, n = 6, 40
    A = np.random.default_rng(5).standard_normal((13, n))
    R = kerdock.representation_definition(A, k).reshape(-1, 13)
    for l in [0, 1, 63, 64, 700, 2047, 2048, 2048 + 39, 2048 + 40, R.shape[0] - 1]:
        np.testing.assert_allclose(kerdock.representation_row(A, l, k), R[l], atol=1e-12)
