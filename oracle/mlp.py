"""FP64 reference of the learned-proposal network -- oracle.

Test infrastructure only (see ``oracle/__init__``).  Not in the paper: the
learned proposal is a project form that ranks candidate indices of Algorithm
1's top-S step from a cheap sketch.  The network is a three-layer perceptron
  H1 = relu(X W1^T + b1),  H2 = relu(H1 W2^T + b2),  Z = H2 W3^T + b3,
trained with binary cross-entropy on logits (positive weight w+),
  loss = (1/B) sum_{b,o} [ w+ y log(1 + e^-z) + (1 - y) log(1 + e^z) ],
and AdamW (Loshchilov & Hutter, decoupled weight decay):
  m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
  p -= lr ( m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps) + wd p ).
relu'(0) is taken as 0.  Parameters are a dict W1, b1, W2, b2, W3, b3.
"""
import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def forward(P, X):
    X = np.asarray(X, dtype=np.float64)
    A1 = X @ P["W1"].T + P["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(A2, 0.0)
    Z = H2 @ P["W3"].T + P["b3"]
    return Z, (X, H1, H2)


def softplus(t):
    return np.logaddexp(0.0, t)


def bce_loss(Z, Y, pos_weight):
    B = Z.shape[0]
    return float((pos_weight * Y * softplus(-Z) + (1.0 - Y) * softplus(Z)).sum() / B)


def bce_grad(Z, Y, pos_weight):
    """d loss / d Z."""
    B = Z.shape[0]
    sig = 1.0 / (1.0 + np.exp(-Z))
    return (pos_weight * Y * (sig - 1.0) + (1.0 - Y) * sig) / B


def backward(P, cache, dZ):
    X, H1, H2 = cache
    g = {}
    g["W3"] = dZ.T @ H2
    g["b3"] = dZ.sum(axis=0)
    dH2 = (dZ @ P["W3"]) * (H2 > 0)
    g["W2"] = dH2.T @ H1
    g["b2"] = dH2.sum(axis=0)
    dH1 = (dH2 @ P["W2"]) * (H1 > 0)
    g["W1"] = dH1.T @ X
    g["b1"] = dH1.sum(axis=0)
    return g


def loss_and_grads(P, X, Y, pos_weight):
    Z, cache = forward(P, X)
    return bce_loss(Z, Y, pos_weight), backward(P, cache, bce_grad(Z, Y, pos_weight))


def adamw_step(P, G, M, V, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update (t = 1 for the first step); returns new (P, M, V)."""
    newP, newM, newV = {}, {}, {}
    for k in NAMES:
        m = beta1 * M[k] + (1 - beta1) * G[k]
        v = beta2 * V[k] + (1 - beta2) * G[k] ** 2
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        newP[k] = P[k] - lr * (mhat / (np.sqrt(vhat) + eps) + wd * P[k])
        newM[k], newV[k] = m, v
    return newP, newM, newV
