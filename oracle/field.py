"""Finite-field construction of the Kerdock set (Sec. 3, Prop. 5) -- oracle.

Test infrastructure only (see ``oracle/__init__``).  Plain Python integers.

Conventions (the paper leaves both open; these readings are shared with the
CUDA library as an interface, not as code):

* GF(2^f), f = k - 1, is polynomial arithmetic over F_2 modulo a fixed
  irreducible polynomial; an element is an integer whose bit j is the
  coefficient of t^j.  For f = 1 the field is F_2 itself.
* The basis B of V = GF(2^f) x F_2 chosen in Prop. 5 is
  B_a = (t^a, 0) for a < f and B_f = (0, 1).  Hence a point p of F_2^k is an
  integer whose bits 0..f-1 hold the field coordinates and whose bit f holds
  the F_2 coordinate alpha.
"""

# Irreducible polynomials of degree f (bit j = coefficient of t^j).
# Sec. 3 only needs *a* field of order 2^(k-1); the choice is an interface
# reading.  Their irreducibility is checked exhaustively in the tests.
IRREDUCIBLE_POLY = {
    1: 0b11,             # t + 1 (F_2; never used for reduction)
    3: 0b1011,           # t^3 + t + 1
    5: 0b100101,         # t^5 + t^2 + 1
    7: 0b10000011,       # t^7 + t + 1
    9: 0b1000010001,     # t^9 + t^4 + 1
    11: 0b100000000101,  # t^11 + t^2 + 1
}


def gf_mul(a, b, f):
    """Product of two elements of GF(2^f) (schoolbook carry-less product,
    then reduction modulo the degree-f polynomial)."""
    poly = IRREDUCIBLE_POLY[f]
    prod = 0
    for j in range(f):
        if (b >> j) & 1:
            prod ^= a << j
    for j in range(2 * f - 2, f - 1, -1):
        if (prod >> j) & 1:
            prod ^= poly << (j - f)
    return prod


def gf_trace(z, f):
    """Field trace tr: GF(2^f) -> F_2, tr(z) = z + z^2 + z^4 + ... + z^(2^(f-1))
    (Sec. 3, before Prop. 5).  Returns 0 or 1."""
    acc = 0
    power = z
    for _ in range(f):
        acc ^= power
        power = gf_mul(power, power, f)
    assert acc in (0, 1), "trace must land in the prime field"
    return acc


def L_map(s, x, alpha, f):
    """The linear map L_s of Prop. 5:
    L_s(x, alpha) = (s^2 x + s tr(sx) + alpha s, tr(sx))."""
    sx = gf_mul(s, x, f)
    t = gf_trace(sx, f)
    first = gf_mul(gf_mul(s, s, f), x, f)
    if t:
        first ^= s
    if alpha:
        first ^= s
    return first, t


def bilinear(u, v, f):
    """The bilinear form of Prop. 5: (x, alpha).(y, beta) = tr(xy) + alpha*beta."""
    (x, alpha), (y, beta) = u, v
    return gf_trace(gf_mul(x, y, f), f) ^ (alpha & beta)


def basis_of_V(f):
    """The basis B of V = GF(2^f) x F_2 fixed above: (t^a, 0) for a < f, then (0, 1)."""
    return [(1 << a, 0) for a in range(f)] + [(0, 1)]


def kerdock_matrix(s, k):
    """(M_s)_{a,c} = B_a . L_s(B_c) (Prop. 5), as a k x k list of 0/1."""
    f = k - 1
    B = basis_of_V(f)
    images = [L_map(s, x, alpha, f) for (x, alpha) in B]
    return [[bilinear(B[a], images[c], f) for c in range(k)] for a in range(k)]


def quadratic_form(M, p):
    """Q_M(p) = p^T M~ p with M~ the strictly upper triangle of M (Sec. 3).
    p is an integer whose bit a is the coordinate p_a."""
    k = len(M)
    q = 0
    for a in range(k):
        if not (p >> a) & 1:
            continue
        for c in range(a + 1, k):
            if (p >> c) & 1:
                q ^= M[a][c]
    return q


def kerdock_sign_bits(k):
    """For every field element s (integer code b in [0, 2^(k-1))) the list of
    Q_{M_s}(p) over p in [0, 2^k): bit 1 means the diagonal entry of D_{M_s}
    in Lemma 6 is -1."""
    d = 1 << k
    out = []
    for s in range(1 << (k - 1)):
        M = kerdock_matrix(s, k)
        out.append([quadratic_form(M, p) for p in range(d)])
    return out


def rank_gf2(M):
    """Rank over F_2 of a 0/1 matrix (Gaussian elimination)."""
    rows = [int("".join(str(v) for v in row), 2) for row in M]
    rank = 0
    ncols = len(M[0]) if M else 0
    for col in range(ncols - 1, -1, -1):
        pivot = None
        for r in range(rank, len(rows)):
            if (rows[r] >> col) & 1:
                pivot = r
                break
        if pivot is None:
            continue
        rows[rank], rows[pivot] = rows[pivot], rows[rank]
        for r in range(len(rows)):
            if r != rank and (rows[r] >> col) & 1:
                rows[r] ^= rows[rank]
        rank += 1
    return rank


def k_for_dimension(n):
    """Smallest even k with d = 2^k >= n (Lemma 6 needs k even; Algorithm 1's
    'power of 2' is read as 'power of 4', see the design notes)."""
    if n < 1:
        raise ValueError("n must be positive")
    k = 2
    while (1 << k) < n:
        k += 2
    return k
