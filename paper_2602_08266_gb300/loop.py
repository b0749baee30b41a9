"""The closed next-best-view loop on synthetic scenes (Sec. III: select the
view of highest information gain, observe it, refine the map, repeat).

Each iteration: score every remaining candidate against the views observed
so far (exactly, or pre-scored by a trained nbv_mlp and pruned), take the
argmax (Eq. 5), render the "observation" of that view from the ground-truth
scene, add it to the observed set, and refine the map with Adam steps on
L1 colour + L1 depth + object cross-entropy over all observed views through
the library's differentiable renderer. Every rendering, score and gradient
runs in the library's kernels; this module only sequences them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class LoopStep:
    chosen: int                 # index into the original candidate list
    score: float                # its normalised total score (Eq. 11)
    loss_before: float          # refinement loss over the observed views
    loss_after: float
    held_out_error: float       # mean L1 colour error of the map on the held-out views


@dataclass
class LoopResult:
    steps: list = field(default_factory=list)
    initial_held_out_error: float = 0.0


def _cams_subset(S, cams, idx):
    idx = np.asarray(idx, np.int64)
    return S.Cameras(cams.R[idx].copy(), cams.t[idx].copy(), cams.fx[idx].copy(), cams.fy[idx].copy(),
                     cams.cx[idx].copy(), cams.cy[idx].copy(), cams.width[idx].copy(), cams.height[idx].copy())


def run(P, S, truth, init, train, cand, held_out, iterations=3, refine_steps=10, lr=2e-3, target=-1,
        mlp=None, keep=64, on_choice=None):
    """truth / init: nbv_synth.Scene (ground truth, starting map); train:
    the initially observed cameras; cand: candidate cameras; held_out:
    cameras the map is evaluated on. on_choice(map_scene, observed, remaining,
    chosen, scores), if given, is called at every choice with the map that
    was scored (an nbv_synth.Scene copy), the observed cameras, the remaining
    candidates' indices, the chosen index and the exact scores [n, 4] of the
    remaining candidates (None when an MLP pruned them). Returns a LoopResult."""
    import torch

    from . import diff
    K, deg = init.K, init.sh_degree
    gt = P.NBVScorer(K, deg)
    gt.load_scene(truth)
    sc = P.NBVScorer(K, deg, batched=1)
    params = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().requires_grad_(True)
              for a in (init.means, init.log_scales, init.quats, init.opacity, init.sh, init.obj_logits)]
    opt = torch.optim.Adam(params, lr=lr)

    def observe(cams):
        out = []
        for i in range(cams.n):
            r = gt.render_camera(cams, i)
            out.append(dict(rgb=r["rgb"], depth=r["depth"], ids=r["obj"].argmax(-1, keepdim=True)))
        return out

    def loss(cams, obs):
        L = 0.0
        for i in range(cams.n):
            rgb, depth, alpha, obj = diff.render(sc, cams, i, *params)
            ce = -(torch.log(obj.clamp_min(1e-6)).gather(-1, obs[i]["ids"])).mean()
            L = L + (rgb - obs[i]["rgb"]).abs().mean() + (depth - obs[i]["depth"]).abs().mean() + 0.1 * ce
        return L / cams.n

    held_obs = observe(held_out)

    def held_error():
        with torch.no_grad():
            sc.load_gaussians(*[p.detach() for p in params])
            e = [float((sc.render_camera(held_out, i)["rgb"] - held_obs[i]["rgb"]).abs().mean())
                 for i in range(held_out.n)]
        return float(np.mean(e))

    result = LoopResult(initial_held_out_error=held_error())
    observed = train
    obs = observe(observed)
    remaining = list(range(cand.n))
    for _ in range(iterations):
        if not remaining:
            break
        sc.load_gaussians(*[p.detach() for p in params])
        sc.set_train_views(observed)
        sub = _cams_subset(S, cand, remaining)
        sc.set_candidates(sub)
        sc.prepare(target)
        scores = None
        if mlp is not None:
            r = sc.score_pruned(mlp, keep)
            best_local, best_score = r["best"], r["best_score"]
        else:
            scores = sc.score_host()
            best_local = int(np.argmax(scores[:, 3]))
            best_score = float(scores[best_local, 3])
        if on_choice is not None:
            snap = [p.detach().cpu().numpy().copy() for p in params]
            on_choice(S.Scene(*snap, deg, K), observed, list(remaining), remaining[best_local], scores)
        chosen = remaining.pop(best_local)
        new = _cams_subset(S, cand, [chosen])
        observed = S.Cameras(*[np.concatenate([getattr(observed, f), getattr(new, f)])
                               for f in ("R", "t", "fx", "fy", "cx", "cy", "width", "height")])
        obs = obs + observe(new)
        with torch.no_grad():
            l0 = float(loss(observed, obs))
        for _ in range(refine_steps):
            opt.zero_grad()
            L = loss(observed, obs)
            L.backward()
            opt.step()
        with torch.no_grad():
            l1 = float(loss(observed, obs))
        result.steps.append(LoopStep(chosen=chosen, score=best_score, loss_before=l0, loss_after=l1,
                                     held_out_error=held_error()))
    sc.close()
    gt.close()
    return result
