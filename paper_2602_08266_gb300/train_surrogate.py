"""Training and evaluation of the learned candidate pre-scorer at scale.

    python -m paper_2602_08266_gb300.train_surrogate --out-dir DIR \
        [--workload surrogate --train-scenes 100 --train-views 250 \
         --eval-scenes 100 --eval-views 1024 --keep 32]

Labels: for every training scene (seeded workload, seeds 1000 + i), the
exact normalised, weighted scores (Eq. 11) of its candidates from the
library's multi-view path, with the candidates' descriptors. Training: the
library's BF16 tensor-core MLP, its own backward and Adam, on
exp(2 z) / 4 of each scene's standardised scores (surrogate.rank_target).
Evaluation on unseen scenes (seeds 20000 + i): the exact scores of all
candidates (the unpruned multi-view path), the MLP's prediction from the
descriptors, the `keep` best predictions kept; the pruned choice is the
exact best among the kept ones (what nbv_score_pruned returns), compared
with the exact best among all. Timings (CUDA events, L2 flushed between
steps) on the first evaluation scene: the pruned step (prepare +
descriptors + MLP + exact scoring of the kept), the unpruned multi-view step
and the per-view path (one launch sequence per candidate), all unprofiled
and over the same candidates.

Writes DIR/surrogate_weights.npz (the network's FP32 parameters) and
DIR/surrogate_report.jsonl (one JSON line per stage and per evaluation
scene, flushed as it goes). Every computation runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np


def _timed(torch, fn, steps, warmup, flush):
    stream = torch.cuda.current_stream()
    out = []
    for i in range(warmup + steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            out.append(e0.elapsed_time(e1))
    return float(np.mean(out))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out-dir", required=True)
    ap.add_argument("--workload", default="surrogate")
    ap.add_argument("--train-scenes", type=int, default=100)
    ap.add_argument("--train-views", type=int, default=250)
    ap.add_argument("--eval-scenes", type=int, default=100)
    ap.add_argument("--eval-views", type=int, default=1024)
    ap.add_argument("--keep", type=int, default=32)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--no-timing", action="store_true")
    ap.add_argument("--weights", default=None,
                    help="evaluate this trained network (a surrogate_weights.npz) instead of training one")
    ap.add_argument("--eval-start", type=int, default=0, help="first evaluation scene (seed 20000 + this)")
    args = ap.parse_args(argv)

    import torch

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import nbv_synth as S
    import paper_2602_08266_gb300 as P
    from paper_2602_08266_gb300 import surrogate as SG

    P.build()
    P.load_library()
    os.makedirs(args.out_dir, exist_ok=True)
    rep = open(os.path.join(args.out_dir, "surrogate_report.jsonl"), "w")

    def log(**kw):
        rep.write(json.dumps(kw) + "\n")
        rep.flush()

    if args.weights:
        w = np.load(args.weights)
        mlp = P.MLP(int(w["d_in"]), int(w["width"]), seed=0)
        mlp.set_params(torch.from_numpy(w["params"]).cuda())
        log(stage="weights", path=os.path.basename(args.weights))
    else:
        # ---- labels
        t0 = time.perf_counter()
        xs, zs = [], []
        for i in range(args.train_scenes):
            wl = S.make_workload(args.workload, seed=1000 + i, n_views=args.train_views)
            x, z, _ = SG.scene_labels(P, wl, target=wl.target)
            xs.append(x)
            zs.append(z)
            if i % 10 == 9:
                log(stage="labels", scenes=i + 1, seconds=round(time.perf_counter() - t0, 1))
        X, Y = torch.cat(xs), SG.rank_target(torch.cat(zs))
        t_labels = time.perf_counter() - t0
        # ---- training
        mlp = P.MLP(P.NBVScorer.DESC_DIM, 256, seed=7)
        t1 = time.perf_counter()
        losses = SG.train(mlp, X, Y, steps=args.steps, batch=args.batch, lr=args.lr)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
        params = mlp.get_params().cpu().numpy()
        np.savez(os.path.join(args.out_dir, "surrogate_weights.npz"), params=params, d_in=P.NBVScorer.DESC_DIM,
                 width=256)
        log(stage="train", labels=int(X.shape[0]), scenes=args.train_scenes, views=args.train_views,
            label_s=round(t_labels, 1), train_s=round(t_train, 1), steps=args.steps, batch=args.batch,
            first_loss=round(losses[0], 4), last_loss=round(losses[-1], 4))
        del X, Y, xs, zs

    # ---- evaluation on unseen scenes
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    agree, ratios, ranks = 0, [], []
    for i in range(args.eval_start, args.eval_start + args.eval_scenes):
        wl = S.make_workload(args.workload, seed=20000 + i, n_views=args.eval_views)
        sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
        sc.load_scene(wl.scene)
        sc.set_train_views(wl.train)
        sc.set_candidates(wl.cand)
        sc.prepare(wl.target)
        full = sc.score_host().astype(np.float64)[:, 3]
        pred = mlp.forward(sc.descriptors()).cpu().numpy().astype(np.float64)
        order = np.argsort(-pred, kind="stable")          # ties to the lower index, as nbv_score_pruned
        kept = order[: args.keep]
        best_exact = int(np.argmax(full))
        best_pruned = int(kept[np.argmax(full[kept])])
        ok = best_pruned == best_exact
        agree += int(ok)
        ratios.append(float(full[best_pruned] / full[best_exact]))
        ranks.append(int(np.nonzero(order == best_exact)[0][0]))
        rec = dict(stage="eval", scene=20000 + i, agree=bool(ok), best_exact=best_exact, best_pruned=best_pruned,
                   score_ratio=round(ratios[-1], 6), rank_of_best=ranks[-1])
        if i == args.eval_start and not args.no_timing:
            out = torch.empty((wl.cand.n, 4), device="cuda")
            rec["pruned_ms"] = _timed(torch, lambda: (sc.prepare(wl.target), sc.score_pruned(mlp, args.keep)), 2, 1,
                                      flush)
            rec["unpruned_ms"] = _timed(torch, lambda: (sc.prepare(wl.target), sc.score(out), sc.argmax()), 1, 1,
                                        flush)
            pv = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=0)
            pv.load_scene(wl.scene)
            pv.set_train_views(wl.train)
            pv.set_candidates(wl.cand)
            rec["per_view_ms"] = _timed(torch, lambda: (pv.prepare(wl.target), pv.score(out), pv.argmax()), 1, 0,
                                        flush)
            pv.close()
        sc.close()
        log(**rec)
    log(stage="summary", eval_scenes=args.eval_scenes, eval_views=args.eval_views, keep=args.keep,
        top1_agreement=agree / max(args.eval_scenes, 1), agree=agree,
        mean_score_ratio=float(np.mean(ratios)) if ratios else None,
        min_score_ratio=float(np.min(ratios)) if ratios else None,
        median_rank_of_best=float(np.median(ranks)) if ranks else None)
    mlp.close()
    rep.close()


if __name__ == "__main__":
    main()
