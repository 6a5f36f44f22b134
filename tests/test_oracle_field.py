"""Pins for the oracle's finite-field / Kerdock-set code (Sec. 3, Prop. 5).

Everything here is checked against facts the paper proves (Prop. 5 (i)-(iii),
the Kerdock-set definition before Prop. 5) or mathematics fixes (field axioms,
trace identities), plus the hand-worked k = 2 case in tests/golden.
"""
import os
import random

import numpy as np
import pytest

from oracle import field

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("f", [1, 3, 5, 7, 9, 11])
def test_polynomial_gives_a_field(f):
    # Every nonzero a satisfies a^(2^f - 1) = 1 iff the quotient ring has no
    # zero divisors, i.e. the polynomial is irreducible.
    for a in range(1, 1 << f):
        acc, base, e = 1, a, (1 << f) - 1
        while e:
            if e & 1:
                acc = field.gf_mul(acc, base, f)
            base = field.gf_mul(base, base, f)
            e >>= 1
        assert acc == 1, (f, a)


@pytest.mark.parametrize("f", [3, 5, 7])
def test_multiplication_is_commutative_associative_distributive(f):
    rng = random.Random(f)
    for _ in range(300):
        a, b, c = (rng.randrange(1 << f) for _ in range(3))
        assert field.gf_mul(a, b, f) == field.gf_mul(b, a, f)
        assert field.gf_mul(field.gf_mul(a, b, f), c, f) == field.gf_mul(a, field.gf_mul(b, c, f), f)
        assert field.gf_mul(a, b ^ c, f) == field.gf_mul(a, b, f) ^ field.gf_mul(a, c, f)


@pytest.mark.parametrize("f", [1, 3, 5, 7, 9, 11])
def test_trace_properties(f):
    # tr is F_2-linear, tr(z^2) = tr(z) (used in the proof of Prop. 5), and tr
    # is onto F_2 with exactly half the field in its kernel.
    rng = random.Random(100 + f)
    elems = range(1 << f) if f <= 7 else [rng.randrange(1 << f) for _ in range(400)]
    ones = 0
    for z in range(1 << f):
        ones += field.gf_trace(z, f)
    assert ones == (1 << f) // 2
    for a in elems:
        assert field.gf_trace(field.gf_mul(a, a, f), f) == field.gf_trace(a, f)
        b = rng.randrange(1 << f)
        assert field.gf_trace(a ^ b, f) == field.gf_trace(a, f) ^ field.gf_trace(b, f)


@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_prop5_facts(k):
    # Prop. 5 proof: (i) (x,a).L_s(x,a) = 0, (ii) L_s is self-adjoint for the
    # form, (iii) L_r(v) = L_s(v) with r != s forces v = 0.
    f = k - 1
    rng = random.Random(k)
    V = [(x, a) for x in range(1 << f) for a in (0, 1)]
    for s in range(1 << f):
        for v in V:
            assert field.bilinear(v, field.L_map(s, v[0], v[1], f), f) == 0
        for _ in range(40):
            u, v = rng.choice(V), rng.choice(V)
            assert (field.bilinear(u, field.L_map(s, v[0], v[1], f), f)
                    == field.bilinear(field.L_map(s, u[0], u[1], f), v, f))
    pairs = [(r, s) for r in range(1 << f) for s in range(1 << f) if r != s]
    if len(pairs) > 400:
        pairs = rng.sample(pairs, 400)
    for r, s in pairs:
        for v in V:
            if field.L_map(r, v[0], v[1], f) == field.L_map(s, v[0], v[1], f):
                assert v == (0, 0)


@pytest.mark.parametrize("k", [2, 4, 6, 8, 10, 12])
def test_kerdock_set_definition(k):
    # Sec. 3: 2^(k-1) symmetric zero-diagonal ("skew-symmetric" over F_2)
    # matrices whose pairwise sums have full rank over F_2.
    f = k - 1
    mats = [field.kerdock_matrix(s, k) for s in range(1 << f)]
    for M in mats:
        A = np.array(M)
        assert (A == A.T).all() and not A.diagonal().any()
    assert len({tuple(map(tuple, M)) for M in mats}) == len(mats)
    rng = random.Random(k)
    pairs = [(r, s) for r in range(len(mats)) for s in range(r + 1, len(mats))]
    if len(pairs) > 3000:
        pairs = rng.sample(pairs, 3000)
    for r, s in pairs:
        S = (np.array(mats[r]) + np.array(mats[s])) % 2
        assert field.rank_gf2(S.tolist()) == k, (r, s)


def test_rank_gf2_brute_force():
    # rank over F_2 equals log2 of the number of distinct row combinations.
    rng = np.random.default_rng(3)
    for _ in range(50):
        M = rng.integers(0, 2, size=(5, 5))
        span = set()
        for mask in range(32):
            v = np.zeros(5, dtype=int)
            for r in range(5):
                if (mask >> r) & 1:
                    v ^= M[r]
            span.add(tuple(v))
        assert 2 ** field.rank_gf2(M.tolist()) == len(span)


def _golden_k2():
    rows = {}
    with open(os.path.join(GOLDEN, "kerdock_n4.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            rows[key] = [[float(t) for t in part.split()] for part in val.split("/")]
    return rows


def test_hand_worked_k2():
    g = _golden_k2()
    assert field.kerdock_matrix(0, 2) == [[int(v) for v in r] for r in g["M0"]]
    assert field.kerdock_matrix(1, 2) == [[int(v) for v in r] for r in g["M1"]]
    for b in (0, 1):
        M = field.kerdock_matrix(b, 2)
        assert [field.quadratic_form(M, p) for p in range(4)] == [int(v) for v in g[f"signs{b}"][0]]


def test_quadratic_form_polarisation():
    # Eq. "polarization": Q(x + y) = Q(x) + x^T M y + Q(y), over random M.
    rng = np.random.default_rng(11)
    k = 6
    for _ in range(20):
        U = np.triu(rng.integers(0, 2, size=(k, k)), 1)
        M = (U + U.T).tolist()
        for _ in range(50):
            x, y = (int(v) for v in rng.integers(0, 1 << k, size=2))
            xv = [(x >> a) & 1 for a in range(k)]
            yv = [(y >> a) & 1 for a in range(k)]
            cross = sum(xv[a] * M[a][c] * yv[c] for a in range(k) for c in range(k)) % 2
            assert field.quadratic_form(M, x ^ y) == (field.quadratic_form(M, x) ^ cross
                                                        ^ field.quadratic_form(M, y))


def test_k_for_dimension():
    assert [field.k_for_dimension(n) for n in (1, 4, 5, 16, 17, 64, 1000, 1024, 2048, 4096)] == \
        [2, 2, 4, 4, 6, 6, 10, 10, 12, 12]
