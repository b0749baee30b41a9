"""Training of the learned candidate pre-scorer (nbv_mlp) on exact scores.

Labels come from the library's own exact path (nbv_score, Eq. 11 totals of
every candidate of a scene); inputs are the library's per-view descriptors.
Within a scene only the ranking of candidates matters for pruning, so each
scene's labels are standardised (zero mean, unit deviation) before
training. Every step of the network runs in the library's kernels (tensor
core layers, hand-written backward, Adam); this module only batches data.
"""
from __future__ import annotations

import numpy as np


def scene_labels(P, wl, target=-1, **cfg):
    """(descriptors [n_cand, 448], standardised exact totals [n_cand], raw
    totals [n_cand]) of one workload, as CUDA tensors."""
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1, **cfg)
    try:
        sc.load_scene(wl.scene)
        sc.set_train_views(wl.train)
        sc.set_candidates(wl.cand)
        sc.prepare(target)
        x = sc.descriptors().clone()
        y = sc.score()[:, 3].clone()
    finally:
        sc.close()
    z = (y - y.mean()) / (y.std() + 1e-12)
    return x, z, y


def rank_target(z):
    """Training target from standardised scores: exp(2 z) / 4 spends the
    network's accuracy on the high-gain candidates that pruning must keep."""
    import torch
    return (torch.exp(2.0 * z) / 4.0).contiguous()


def train(mlp, X, Y, steps=400, batch=512, lr=2e-3, seed=0):
    """Adam steps on random mini-batches of (X, Y); returns the losses."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    n = X.shape[0]
    losses = []
    for i in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g).cuda()
        xb = X[idx].contiguous()
        yb = Y[idx].contiguous()
        want = (i % 20 == 0) or i == steps - 1
        loss = mlp.train_step(xb, yb, lr, want_loss=want)
        if want:
            losses.append(loss)
    return losses
