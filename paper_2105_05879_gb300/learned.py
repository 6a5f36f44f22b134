"""Learned proposal: a network that ranks Algorithm 1's refinement candidates.

Not in the paper.  For a fixed A, the method itself generates training pairs:
a cheap sketch mu (a clone of the plan with small J, K) is the input, and the
support of the full method's thresholded output h_eps(Ax) is the label.  The
network (kerdock_mlp_*, trained on the GPU by the library's own forward,
backward and AdamW kernels) scores every index; the top S' scores are refined
exactly (kerdock_refine_scores).  With the plain top-|mu| ranking as the
fallback, the gain is fewer samples N and fewer refined rows S' for the same
support recall.  Every step runs in the library's CUDA kernels; this module
only orders the calls.
"""
import numpy as np

from . import kerdock as K


class LearnedProposal:
    def __init__(self, plan, J_sketch, K_sketch, S_prime, hidden=512, max_batch=1024, seed=1,
                 feat_scale=None, residual=False):
        self.plan = plan
        self.torch = plan.torch
        m = plan.info["m"]
        self.sketch = plan.clone(J_sketch, K_sketch, 1)  # only mu is used from the sketch
        self.S_prime = int(S_prime)
        self.mlp = K.KerdockMLP(m, hidden, m, max_batch, device=plan.device)
        self.mlp.init(seed)
        # the support does not depend on the signs of Ax, so the network sees |mu|
        self.mlp.set_input(K.KERDOCK_MLP_INPUT_ABS)
        if residual:
            # logits = MLP(|mu|) + |mu| with the last layer zeroed: training starts
            # from the plain top-|mu| ranking and learns corrections to it
            self.mlp.set_skip(1.0)
            W3, b3 = self.mlp.tensors(self.mlp.params)[4:6]
            W3.zero_()
            b3.zero_()
            self.mlp.sync_weights()
        self.feat_scale = feat_scale
        self.max_batch = max_batch

    def sketch_mu(self, X, seed):
        """mu of the reduced-N sketch for every row of X (q x m, float32)."""
        t = self.torch
        q = X.shape[0]
        m = self.plan.info["m"]
        mu = t.empty((q, m), dtype=t.float32, device=self.plan.device)
        for s in range(0, q, 65536):
            e = min(q, s + 65536)
            out = self.sketch.apply(X[s:e], 1.0, seed + s, debug=True)
            mu[s:e].copy_(out[3])
        return mu

    def labels_from_method(self, X, eps, seed):
        """0/1 labels: the support the plain (full-N) method returns for each x."""
        t = self.torch
        q = X.shape[0]
        m = self.plan.info["m"]
        Y = t.zeros((q, m), dtype=t.float32, device=self.plan.device)
        for s in range(0, q, 65536):
            e = min(q, s + 65536)
            idx, val, cnt = self.plan.apply(X[s:e], eps, seed + s)
            S = idx.shape[1]
            valid = t.arange(S, device=idx.device)[None, :] < cnt[:, None]
            rows = t.arange(e - s, device=idx.device)[:, None].expand(-1, S)
            Y[s:e][rows[valid], idx[valid].long()] = 1.0
        return Y

    def train(self, mu, Y, epochs=3, batch=1024, lr=2e-3, pos_weight=None, wd=1e-4, seed=0,
              log=None):
        t = self.torch
        q = mu.shape[0]
        if self.feat_scale is None:
            self.feat_scale = float(1.0 / (mu.abs().mean().item() + 1e-12))
        if pos_weight is None:
            frac = float(Y.mean().item())
            pos_weight = float(np.clip((1 - frac) / max(frac, 1e-6), 1.0, 100.0)) ** 0.5
        gen = t.Generator(device="cpu").manual_seed(seed)
        batch = min(batch, self.max_batch)
        losses = []
        for ep in range(epochs):
            perm = t.randperm(q, generator=gen).to(mu.device)
            for s in range(0, q - batch + 1, batch):
                ix = perm[s:s + batch]
                xb = mu.index_select(0, ix).contiguous()
                yb = Y.index_select(0, ix).contiguous()
                self.mlp.backward(xb, yb, self.feat_scale, pos_weight)
                self.mlp.adamw(lr, wd=wd)
            losses.append(self.mlp.loss())
            if log:
                log(f"epoch {ep}: loss {losses[-1]:.4f}")
        return losses

    def scores(self, mu):
        t = self.torch
        q = mu.shape[0]
        out = t.empty_like(mu)
        for s in range(0, q, self.max_batch):
            e = min(q, s + self.max_batch)
            self.mlp.forward(mu[s:e].contiguous(), self.feat_scale, out[s:e])
        return out

    def apply(self, X, eps, seed, flags=0):
        """Learned pipeline: sketch -> network scores -> top S' refine -> threshold."""
        mu = self.sketch_mu(X, seed)
        sc = self.scores(mu)
        return self.plan.refine_scores(X, sc, self.S_prime, eps, flags)

    def launches_per_apply(self, q):
        """Library kernels one apply(q) launches: one sketch query kernel per
        65536 rows, four network kernels (input conversion, three layers) per
        max_batch rows, one refinement kernel."""
        return -(-q // 65536) + 4 * -(-q // self.max_batch) + 1

    def apply_plain_sketch(self, X, eps, seed, flags=0):
        """The fallback with the same budget: sketch -> top S' of |mu| -> refine."""
        mu = self.sketch_mu(X, seed)
        return self.plan.refine_scores(X, mu.abs(), self.S_prime, eps, flags)


def support_recall(idx, cnt, truth):
    """Fraction of true support entries found, and fraction of queries recovered exactly."""
    idx = idx.cpu().numpy()
    cnt = cnt.cpu().numpy()
    hit = tot = exact = 0
    for r, tr in enumerate(truth):
        got = set(idx[r, :cnt[r]].tolist())
        trs = set(tr.tolist())
        hit += len(got & trs)
        tot += len(trs)
        exact += got == trs
    return hit / max(tot, 1), exact / max(len(truth), 1)
