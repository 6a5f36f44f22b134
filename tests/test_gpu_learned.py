"""Learned proposal: the library's bfloat16 MLP kernels against the FP64
oracle (oracle/mlp.py), the score-ranked refinement against its definition,
and what the trained network gains over the plain top-|mu| ranking at the same
sketch size and refinement budget."""
import math

import numpy as np
import pytest

from gpu_common import build_and_load, f32, oq, torch_cuda
from oracle import mlp as omlp
import workloads

pytestmark = pytest.mark.gpu


def bf16_round(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).bfloat16().float().numpy().astype(np.float64)


def _small_net(K, torch, seed=3, dims=(64, 32, 48), B=16):
    net = K.KerdockMLP(*dims, max_batch=B)
    net.init(seed)
    torch.cuda.synchronize()
    return net


def _params_np(net):
    return {k: v.detach().cpu().numpy().astype(np.float64)
            for k, v in zip(omlp.NAMES, net.tensors(net.params))}


def test_mlp_forward_backward_vs_oracle():
    torch = torch_cuda()
    K = build_and_load()
    B = 16
    net = _small_net(K, torch, B=B)
    rng = np.random.default_rng(0)
    feats = rng.standard_normal((B, 64)).astype(np.float32)
    labels = (rng.random((B, 48)) < 0.2).astype(np.float32)
    scale, pw = 0.7, 3.0
    ft = torch.from_numpy(feats).cuda()
    lt = torch.from_numpy(labels).cuda()
    logits = net.forward(ft, scale).cpu().numpy()
    net.backward(ft, lt, scale, pw)
    loss = net.loss()
    gpu_grads = {k: v.detach().cpu().numpy().astype(np.float64)
                 for k, v in zip(omlp.NAMES, net.tensors(net.grads))}
    # the oracle on the values the GPU multiplies: bf16 weights and features
    P = _params_np(net)
    for k in ("W1", "W2", "W3"):
        P[k] = bf16_round(P[k])
    X = bf16_round(scale * feats)
    Z, _ = omlp.forward(P, X)
    # each bf16 rounding of an activation changes it by <= 2^-8 relatively
    np.testing.assert_allclose(logits, Z, rtol=0, atol=0.03 * np.abs(Z).max() + 1e-3)
    ref_loss, G = omlp.loss_and_grads(P, X, labels.astype(np.float64), pw)
    assert abs(loss - ref_loss) <= 0.02 * abs(ref_loss) + 1e-4
    for k in omlp.NAMES:
        err = np.abs(gpu_grads[k] - G[k]).max()
        assert err <= 0.05 * np.abs(G[k]).max() + 1e-5, (k, err, np.abs(G[k]).max())
    net.close()


def test_mlp_adamw_vs_oracle():
    torch = torch_cuda()
    K = build_and_load()
    net = _small_net(K, torch, seed=5)
    rng = np.random.default_rng(1)
    # install known gradients and run two steps against the oracle's AdamW
    P = _params_np(net)
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    for t in (1, 2):
        G = {k: rng.standard_normal(v.shape) for k, v in P.items()}
        for dst, k in zip(net.tensors(net.grads), omlp.NAMES):
            dst.copy_(torch.from_numpy(G[k].astype(np.float32)))
        G = {k: v.astype(np.float32).astype(np.float64) for k, v in G.items()}
        net.adamw(1e-2, 0.9, 0.999, 1e-8, 0.05)
        P, M, V = omlp.adamw_step(P, G, M, V, t, 1e-2, 0.9, 0.999, 1e-8, 0.05)
        got = _params_np(net)
        for k in omlp.NAMES:
            np.testing.assert_allclose(got[k], P[k], rtol=1e-5, atol=1e-6)
    net.close()


def test_refine_scores_definition():
    torch = torch_cuda()
    K = build_and_load()
    n = 256
    A = workloads.random_orthogonal(n, 8).astype(np.float32)
    plan = K.KerdockPlan(n, n, J=4, K=2, S=4)
    plan.preprocess(torch.from_numpy(A).cuda())
    rng = np.random.default_rng(2)
    X = rng.standard_normal((9, n)).astype(np.float32)
    sc = rng.standard_normal((9, n)).astype(np.float32)
    sc[3, 10:20] = 5.0  # ties: smaller indices first
    S = 13
    idx, val, cnt = plan.refine_scores(torch.from_numpy(X).cuda(), torch.from_numpy(sc).cuda(), S, 0.0,
                                       flags=1)
    plan.sync()
    idx, val, cnt = idx.cpu().numpy(), val.cpu().numpy(), cnt.cpu().numpy()
    for q in range(9):
        order = sorted(range(n), key=lambda i: (-sc[q, i], i))[:S]
        np.testing.assert_array_equal(idx[q, :cnt[q]], np.sort(order))
        np.testing.assert_allclose(val[q, :cnt[q]], f32(A)[np.sort(order)] @ f32(X[q]), atol=1e-5)
    plan.close()


def test_learned_proposal_gains_over_plain_ranking():
    # Structured supports (2 runs of 4 consecutive indices): with a sketch of
    # only N = 16 samples and S' = 24 refined rows, the network trained on
    # 100k method-generated pairs recovers more of h_eps(Ax) than ranking by |mu|.
    torch = torch_cuda()
    K = build_and_load()
    from paper_2105_05879_gb300.learned import LearnedProposal, support_recall
    n, s = 256, 8
    amp, eps = 1 / math.sqrt(s), 0.5 / math.sqrt(s)
    A = workloads.random_orthogonal(n, 12).astype(np.float32)
    plan = K.KerdockPlan(n, n, J=200, K=2, S=10 * s)
    plan.preprocess(torch.from_numpy(A).cuda())

    def queries(q, seed):
        Z = workloads.sparse_codes(n, q, s, amp, seed, blocks=(2, 4))
        return torch.from_numpy((Z @ f32(A)).astype(np.float32)).cuda(), Z

    lp = LearnedProposal(plan, J_sketch=8, K_sketch=2, S_prime=24, hidden=512, max_batch=1024,
                         seed=4)
    Xtr, _ = queries(100000, 100)
    mu = lp.sketch_mu(Xtr, 7)
    Y = lp.labels_from_method(Xtr, eps, 9)
    losses = lp.train(mu, Y, epochs=6, batch=512, lr=1e-3, seed=0)
    assert losses[-1] < losses[0]
    Xev, Zev = queries(4000, 200)
    truth = [np.nonzero(np.abs(z) >= eps)[0] for z in Zev]
    li, lv, lc = lp.apply(Xev, eps, 11)
    pi, pv, pc = lp.apply_plain_sketch(Xev, eps, 11)
    plan.sync()
    rec_l, ex_l = support_recall(li, lc, truth)
    rec_p, ex_p = support_recall(pi, pc, truth)
    print(f"learned recall {rec_l:.3f} exact {ex_l:.3f} | plain-sketch recall {rec_p:.3f} exact {ex_p:.3f}")
    # measured on a GB300: learned 0.55 vs plain 0.37 (the network sees |mu| and
    # learns the two-run support structure from the method's own outputs)
    assert rec_l >= rec_p + 0.10
    plan.close()
