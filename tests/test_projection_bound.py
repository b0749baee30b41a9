"""The conservative radius bound the multi-view projection uses to drop,
before the rest of its key path, (view, Gaussian) slots whose rectangle
cannot reach the view's box of target tiles: the oracle's radius
ceil(3 sqrt(lambda_max)) of the EWA 2D covariance (Sec. IV-A.2, the 3DGS
projection) never exceeds 3 sqrt(||J||_F^2 s_max^2 + 2 dilation + 0.5) * 1.01
+ 2 pixels, less one pixel of slack, on isotropic, elongated and flat
Gaussians anywhere in and around the view (guard-band clamping included)."""
import numpy as np
import pytest

import nbv_synth as S
from helpers import make_scene
from oracle import oracle as O


def _bound(scene, cams, v, hp):
    R, t = cams.R[v].astype(np.float64), cams.t[v].astype(np.float64)
    fx, fy = float(cams.fx[v]), float(cams.fy[v])
    W, H = float(cams.width[v]), float(cams.height[v])
    p = scene.means.astype(np.float64) @ R.T + t
    tz = p[:, 2]
    limx, limy = hp.guard * 0.5 * W / fx, hp.guard * 0.5 * H / fy
    xz = np.clip(p[:, 0] / tz, -limx, limx)
    yz = np.clip(p[:, 1] / tz, -limy, limy)
    smax = np.exp(scene.log_scales.astype(np.float64)).max(1)
    tr = (fx * fx * (1 + xz * xz) + fy * fy * (1 + yz * yz)) / (tz * tz) * smax * smax + 2 * hp.dilation
    return 3.0 * np.sqrt(tr + 0.5) * 1.01 + 2.0


def _check(scene, cams):
    o = O.OracleScene(scene)
    n_checked = 0
    for v in range(cams.n):
        pr = o.project32(cams, v)
        ok = pr["rect"][:, 0] >= 0
        rb = _bound(scene, cams, v, o.hyper)
        r = pr["radius"].astype(np.float64)
        assert np.all(r[ok] <= rb[ok] - 1.0), (v, float(np.max(r[ok] - rb[ok])))
        n_checked += int(ok.sum())
    return n_checked


def test_bound_on_the_tiny_workload():
    wl = S.make_workload("tiny")
    assert _check(wl.scene, wl.cand) > 1000


def test_bound_on_a_reduced_tabletop_scene():
    wl = S.make_workload("batch", n_views=6, scale=0.02)
    assert _check(wl.scene, wl.cand) > 1000


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bound_on_elongated_flat_and_off_screen_gaussians(seed):
    rng = np.random.default_rng(seed)
    n = 4000
    means = rng.uniform(-0.6, 0.6, (n, 3))
    # anisotropy up to ~e^5 between the axes: needles, discs and blobs
    log_scales = np.log(0.01) + rng.normal(0, 1.2, (n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    scene = make_scene(means, log_scales, q)
    cams = S.sphere_cameras(rng, 4, 0.9, 320, 240, 262.5)
    assert _check(scene, cams) > 1000
