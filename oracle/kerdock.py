"""Kerdock mutually unbiased bases and the representation {A s_l} -- oracle.

Test infrastructure only (see ``oracle/__init__``).  float64 numpy.

Indexing (shared with the CUDA library as an interface):
  d = 2^k (k even), number of bases B = d/2 + 1, design size L = d*B.
  Basis index b in [0, d/2) is the Kerdock basis of the field element whose
  integer code is b; b = d/2 is the identity basis.  Sample index l = b*d + w.
  The representation is stored as R[b, w, i] = (A s_{b,w})_i.
"""
import numpy as np

from . import field


def point_bits(k, n=None):
    """(n, k) 0/1 array: row p holds the coordinates p_a = bit a of p."""
    d = 1 << k
    p = np.arange(d if n is None else n)
    return (p[:, None] >> np.arange(k)[None, :]) & 1


def sign_row(b, k, n=None):
    """Q_{M_b}(p) = p^T M~_b p mod 2 for p < n (default n = d): Lemma 6 step (i),
    with M~ the strictly upper triangle of the Kerdock matrix M_b (Sec. 3)."""
    M = np.array(field.kerdock_matrix(b, k), dtype=np.int64)
    Mup = np.triu(M, 1)
    P = point_bits(k, n)
    return ((P @ Mup) * P).sum(axis=1) % 2


def sign_matrix(k):
    """(d/2) x d array of Q_{M_b}(p) in {0,1} (Lemma 6 step (i))."""
    return np.stack([sign_row(b, k) for b in range((1 << k) // 2)])


def walsh_matrix(k):
    """W[w, p] = (-1)^(w^T p) over F_2^k; W = sqrt(d) H^{(x)k} (Lemma 6)."""
    d = 1 << k
    idx = np.arange(d)
    par = np.zeros((d, d), dtype=np.int64)
    for bit in range(k):
        par ^= ((idx[:, None] >> bit) & 1) & ((idx[None, :] >> bit) & 1)
    return 1.0 - 2.0 * par


def mub_vectors(k):
    """All L = d(d/2+1) unit vectors of the projective 2-design as an L x d
    array, row l = b*d + w.  Rows b < d/2 follow Eq. "definition of vectors":
    u_{M,w}(p) = 2^(-k/2) (-1)^(Q_M(p) + w^T p); the last d rows are the
    identity basis e_w (Sec. 3, after Prop. 4)."""
    d = 1 << k
    Q = sign_matrix(k)                      # (d/2, d)
    W = walsh_matrix(k)                     # (d, d)
    U = np.empty((d // 2 + 1, d, d))
    for b in range(d // 2):
        U[b] = W * (1.0 - 2.0 * Q[b])[None, :] / np.sqrt(d)
    U[d // 2] = np.eye(d)
    return U.reshape(-1, d)


def sample_vectors(n, k):
    """Rows s_l = sqrt(d) Pi u_l, Pi = projection onto the first n coordinates
    (Algorithm 1, preprocessing step).  Shape L x n."""
    d = 1 << k
    if n > d:
        raise ValueError("n must not exceed d")
    return np.sqrt(d) * mub_vectors(k)[:, :n]


def sample_vector(l, n, k):
    """One sample vector s_l without building the design (for large d)."""
    d = 1 << k
    b, w = divmod(int(l), d)
    if b == d // 2:
        s = np.zeros(n)
        if w < n:
            s[w] = np.sqrt(d)
        return s
    q = sign_row(b, k, n)
    p = np.arange(n)
    wp = np.zeros(n, dtype=np.int64)
    for bit in range(k):
        wp ^= ((w >> bit) & 1) & ((p >> bit) & 1)
    return 1.0 - 2.0 * (q ^ wp)


def representation_definition(A, k):
    """R[l, :] = A s_l by its definition (Algorithm 1: 'compute {A s_l}'),
    one dense product per sample vector.  Returns shape (B, d, m)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    d = 1 << k
    S = sample_vectors(n, k)                # (L, n)
    R = S @ A.T                             # (L, m): row l = (A s_l)^T
    return R.reshape(d // 2 + 1, d, m)


def fwht_rows(X):
    """Unnormalised fast Walsh-Hadamard transform along the last axis:
    Y[..., w] = sum_p X[..., p] (-1)^(w^T p).  Textbook butterflies."""
    Y = np.array(X, dtype=np.float64, copy=True)
    d = Y.shape[-1]
    h = 1
    while h < d:
        Y = Y.reshape(Y.shape[:-1] + (d // (2 * h), 2, h))
        lo = Y[..., 0, :].copy()
        hi = Y[..., 1, :].copy()
        Y[..., 0, :] = lo + hi
        Y[..., 1, :] = lo - hi
        Y = Y.reshape(Y.shape[:-3] + (d,))
        h *= 2
    return Y


def representation_lemma6(A, k, bases=None):
    """The fast preprocessing of Lemma 6, step by step:
    for each Kerdock matrix M: (i) signs (-1)^(Q_M(x)); (ii) FWHT of each row
    (Pi^* a_i)^T D_M; (iii) the product with sqrt(d) H^{(x)k} = W gives the
    columns A s_{M,w}; finally the identity basis gives sqrt(d) A e_w.
    Returns shape (len(bases), d, m); by default all B bases."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    d = 1 << k
    if bases is None:
        bases = range(d // 2 + 1)
    bases = list(bases)
    Apad = np.zeros((m, d))
    Apad[:, :n] = A                         # Pi^* a_i
    out = np.empty((len(bases), d, m))
    for t, b in enumerate(bases):
        if b == d // 2:
            out[t] = np.sqrt(d) * Apad.T    # sqrt(d) A Pi e_w: zero for w >= n
        else:
            signed = Apad * (1.0 - 2.0 * sign_row(b, k))[None, :]
            out[t] = fwht_rows(signed).T    # row w holds (A s_{b,w})^T
    return out


def representation_row(A, l, k):
    """One row A s_l of the representation, computed lazily (used where the
    full representation does not fit in host memory)."""
    A = np.asarray(A, dtype=np.float64)
    return A @ sample_vector(l, A.shape[1], k)
