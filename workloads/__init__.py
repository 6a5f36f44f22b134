"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws inputs; it holds none of the method's arithmetic.  The
recipe follows Sec. 4 of the paper: A is a random orthogonal matrix, and each
query is x = A^T z for a sparse code z, so that Ax = z ("straightforward since
A^{-1} = A^T").  Everything is float64 here; callers hand float32 copies to the
GPU and float64 copies of those float32 values to the oracle.
"""
from dataclasses import dataclass, field
import math

import numpy as np


def random_orthogonal(n, seed):
    """Orthogonal n x n matrix from the QR factorisation of a seeded N(0,1)
    matrix, with the signs of R's diagonal moved into Q (Haar measure)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q *= np.sign(np.diag(R))[None, :]
    return Q


def sparse_codes(n, q, s, amp, seed, noise=0.0, blocks=None):
    """q codes z in R^n, each with s nonzeros of magnitude amp and random
    signs.  blocks=None: support uniform without replacement; blocks=(nb, bl):
    nb non-overlapping contiguous runs of length bl (nb * bl == s) at random
    offsets.  noise > 0 adds N(0, noise^2) to every entry."""
    rng = np.random.default_rng(seed)
    Z = np.zeros((q, n))
    for r in range(q):
        if blocks is None:
            supp = rng.choice(n, size=s, replace=False)
        else:
            nb, bl = blocks
            assert nb * bl == s
            supp = _block_support(rng, n, nb, bl)
        Z[r, supp] = amp * rng.choice([-1.0, 1.0], size=s)
    if noise > 0:
        Z += noise * rng.standard_normal((q, n))
    return Z


def _block_support(rng, n, nb, bl):
    # Choose nb non-overlapping runs: place them in n - nb*bl free slots.
    free = n - nb * bl
    gaps = np.sort(rng.choice(free + nb, size=nb, replace=False))
    starts = gaps - np.arange(nb) + np.arange(nb) * bl
    return np.concatenate([np.arange(st, st + bl) for st in starts])


def queries_from_codes(A, Z):
    """Rows x = A^T z, i.e. X = Z A."""
    return np.asarray(Z) @ np.asarray(A)


@dataclass
class Workload:
    name: str
    n: int
    m: int
    queries: int
    s: int
    amp: float
    eps: float
    noise: float = 0.0
    blocks: tuple = None
    seed: int = 0
    J: int = 0
    K: int = 2
    S: int = 0
    dtype: str = "f32"
    extra: dict = field(default_factory=dict)

    @property
    def seed_A(self):
        return self.seed

    @property
    def seed_queries(self):
        return self.seed + 1

    @property
    def seed_apply(self):
        return self.seed + 2

    def make_A(self):
        assert self.m == self.n
        return random_orthogonal(self.n, self.seed_A)

    def make_codes(self, q=None, offset_seed=0):
        return sparse_codes(self.n, q or self.queries, self.s, self.amp,
                            self.seed_queries + offset_seed, self.noise, self.blocks)


# The five synthetic workloads (sizes, distributions and thresholds follow the
# paper's Sec. 4 recipe scaled to n = 64 ... 4096).  J is the batch size of the
# median of means; S = min(10 s, m) as in Sec. 4.
WORKLOADS = {
    "n64": Workload("n64", 64, 64, 100, 4, 0.5, 0.25, J=64, K=2, S=40),
    "n1024": Workload("n1024", 1024, 1024, 1000, 16, 0.25, 0.125, noise=1e-3,
                      J=375, K=2, S=160),
    "n4096_bf16": Workload("n4096_bf16", 4096, 4096, 4096, 32, 1 / math.sqrt(32), 0.09,
                           J=1000, K=2, S=320, dtype="bf16"),
    "n2048_blocks": Workload("n2048_blocks", 2048, 2048, 10000, 32, 1 / math.sqrt(32),
                             0.5 / math.sqrt(32), blocks=(4, 8), J=375, K=2, S=320),
}
