"""The model bench.py turns its bounded oracle sample into a step time:
per candidate resolution, two pixel-row strides fix t = a + b / stride, the
whole view costs a + b, the step is the candidates x their resolution's
whole-view time plus the training state as its views x the largest
resolution's whole-view time (scaled by pixels). Checked on synthetic
timings with known a and b, on the batching workload's cameras."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import nbv_synth as S  # noqa: E402


def test_two_stride_model_recovers_whole_view_times():
    wl = S.make_workload("batch", n_views=6, scale=0.01)
    plan = bench.sample_plan(wl)
    # one candidate of each resolution, two strides each, the larger first
    assert len(plan) == 4 and len({v for v, _, _ in plan}) == 2
    px = {v: int(wl.cand.width[v]) * int(wl.cand.height[v]) for v, _, _ in plan}
    ab = {v: (3.0 + 0.5 * i, 40.0 * px[v] / 76800.0) for i, v in enumerate(sorted(px))}
    times = {(v, s): ab[v][0] + ab[v][1] / s for v, _, s in plan}
    t_step, prep_s, per_res = bench.oracle_model(wl, times)
    for v, (full, count, p) in per_res.items():
        assert full == pytest.approx(sum(ab[v]), rel=1e-12)
        assert count == sum(1 for u in range(wl.cand.n)
                            if int(wl.cand.width[u]) * int(wl.cand.height[u]) == p)
    big = max(per_res, key=lambda v: px[v])
    train_px = int(wl.train.width[0]) * int(wl.train.height[0])
    assert prep_s == pytest.approx(wl.train.n * sum(ab[big]) * train_px / px[big], rel=1e-12)
    assert t_step == pytest.approx(prep_s + sum(f * c for f, c, _ in per_res.values()), rel=1e-12)
    assert sum(c for _, c, _ in per_res.values()) == wl.cand.n


def test_one_stride_falls_back_to_row_scaling():
    wl = S.make_workload("batch", n_views=2, scale=0.01)
    plan = bench.sample_plan(wl)
    times = {}
    for v, _, s in plan:
        if (v, s) not in {(u, t) for (u, t) in times} and all(u != v for (u, _) in times):
            times[(v, s)] = 2.0
    _, _, per_res = bench.oracle_model(wl, times)
    for (v, s), t in times.items():
        assert per_res[v][0] == pytest.approx(t * s)
