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


def test_forward_hand_worked_network():
    # A 2 -> 2 -> 2 -> 1 network with integer weights, worked by hand:
    #   x = (1, 2): W1 x + b1 = (1 - 2 + 0, 2 + 2 - 1) = (-1, 3), relu -> (0, 3)
    #               W2 h1 + b2 = (0 + 3 + 1, 0 + 6 + 0) = (4, 6), relu -> (4, 6)
    #               W3 h2 + b3 = 4 - 6 - 1 = -3          (no relu on the logits)
    #   x = (3, 1): (3 - 1, 6 + 1 - 1) = (2, 6) -> (2 + 6 + 1, -2 + 12) = (9, 10)
    #               -> 9 - 10 - 1 = -2
    # A relu on the output layer, a dropped bias or a transposed W1 changes a logit.
    P = {"W1": np.array([[1.0, -1.0], [2.0, 1.0]]), "b1": np.array([0.0, -1.0]),
         "W2": np.array([[1.0, 1.0], [-1.0, 2.0]]), "b2": np.array([1.0, 0.0]),
         "W3": np.array([[1.0, -1.0]]), "b3": np.array([-1.0])}
    Z, (X, H1, H2) = mlp.forward(P, np.array([[1.0, 2.0], [3.0, 1.0]]))
    np.testing.assert_array_equal(Z, [[-3.0], [-2.0]])
    np.testing.assert_array_equal(H1, [[0.0, 3.0], [2.0, 6.0]])
    np.testing.assert_array_equal(H2, [[4.0, 6.0], [9.0, 10.0]])


def test_adamw_bias_correction_over_steps():
    # Constant gradient g from zero moments: m_t = (1 - b1^t) g and
    # v_t = (1 - b2^t) g^2, so the bias-corrected moments are g and g^2 at
    # every t and each step is lr (g / (|g| + eps) + wd p) with p before the
    # step.  A correction by (1 - b) instead of (1 - b^t) fails from t = 2.
    rng = np.random.default_rng(2)
    P = _params(rng, 3, 2, 3)
    G = {k: rng.standard_normal(v.shape) for k, v in P.items()}
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    want = {k: v.copy() for k, v in P.items()}
    b1, b2, lr, eps, wd = 0.9, 0.999, 0.01, 1e-8, 0.05
    for t in range(1, 7):
        P, M, V = mlp.adamw_step(P, G, M, V, t, lr=lr, beta1=b1, beta2=b2, eps=eps, wd=wd)
        for k in mlp.NAMES:
            want[k] = want[k] - lr * (G[k] / (np.abs(G[k]) + eps) + wd * want[k])
            np.testing.assert_allclose(P[k], want[k], rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(M[k], (1 - b1 ** t) * G[k], rtol=1e-12)
            np.testing.assert_allclose(V[k], (1 - b2 ** t) * G[k] ** 2, rtol=1e-12)


def test_adamw_two_steps_by_hand():
    # Scalar p, gradients +1 then -1, b1 = 1/2, b2 = 3/4, lr = 1, eps = wd = 0:
    #   t = 1: m = 1/2, v = 1/4; mhat = 1, vhat = 1           -> p = p0 - 1
    #   t = 2: m = 1/4 - 1/2 = -1/4, v = 3/16 + 1/4 = 7/16;
    #          mhat = (-1/4) / (3/4) = -1/3, vhat = (7/16) / (7/16) = 1 -> p += 1/3
    one = {k: np.ones(1) for k in mlp.NAMES}
    zero = {k: np.zeros(1) for k in mlp.NAMES}
    P = {k: np.full(1, 5.0) for k in mlp.NAMES}
    P, M, V = mlp.adamw_step(P, one, zero, zero, 1, lr=1.0, beta1=0.5, beta2=0.75, eps=0.0)
    P, M, V = mlp.adamw_step(P, {k: -v for k, v in one.items()}, M, V, 2, lr=1.0, beta1=0.5,
                             beta2=0.75, eps=0.0)
    for k in mlp.NAMES:
        assert abs(P[k][0] - (5.0 - 1.0 + 1.0 / 3.0)) < 1e-14
        assert M[k][0] == -0.25 and V[k][0] == 7.0 / 16.0
