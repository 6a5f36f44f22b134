"""Pins for the oracle's learned-proposal network (oracle/mlp.py): analytic
gradients against central finite differences, the BCE closed form at z = 0,
and the first AdamW step's closed form."""
import math

import numpy as np

from oracle import mlp


def _params(rng, i, h, o):
    return {"W1": rng.standard_normal((h, i)) * 0.5, "b1": rng.standard_normal(h) * 0.1,
            "W2": rng.standard_normal((h, h)) * 0.5, "b2": rng.standard_normal(h) * 0.1,
            "W3": rng.standard_normal((o, h)) * 0.5, "b3": rng.standard_normal(o) * 0.1}


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    P = _params(rng, 7, 5, 6)
    X = rng.standard_normal((4, 7))
    Y = (rng.random((4, 6)) < 0.3).astype(float)
    loss, G = mlp.loss_and_grads(P, X, Y, 3.0)
    h = 1e-6
    for k in mlp.NAMES:
        flat = P[k].reshape(-1)
        gflat = G[k].reshape(-1)
        for idx in range(flat.size):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss_and_grads(P, X, Y, 3.0)[0]
            flat[idx] = old - h
            lm = mlp.loss_and_grads(P, X, Y, 3.0)[0]
            flat[idx] = old
            assert abs((lp - lm) / (2 * h) - gflat[idx]) < 1e-6 * max(1.0, abs(gflat[idx])), (k, idx)


def test_bce_closed_forms():
    Z = np.zeros((2, 3))
    Y = np.array([[1.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    # at z = 0 every term is log 2 (times w+ for positives): (1/B) sum
    assert abs(mlp.bce_loss(Z, Y, 2.0) - (3 * 2 * math.log(2) + 3 * math.log(2)) / 2) < 1e-12
    np.testing.assert_allclose(mlp.bce_grad(Z, Y, 2.0), (2.0 * Y * (-0.5) + (1 - Y) * 0.5) / 2)


def test_first_adamw_step_closed_form():
    # t = 1: mhat = g, vhat = g^2, so the step is lr (g/(|g| + eps) + wd p)
    rng = np.random.default_rng(1)
    P = _params(rng, 3, 2, 3)
    G = {k: rng.standard_normal(v.shape) for k, v in P.items()}
    Z0 = {k: np.zeros_like(v) for k, v in P.items()}
    newP, M, V = mlp.adamw_step(P, G, Z0, Z0, 1, lr=0.01, eps=1e-8, wd=0.1)
    for k in mlp.NAMES:
        np.testing.assert_allclose(newP[k], P[k] - 0.01 * (G[k] / (np.abs(G[k]) + 1e-8) + 0.1 * P[k]),
                                   rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(M[k], 0.1 * G[k])
        np.testing.assert_allclose(V[k], 0.001 * G[k] ** 2)
