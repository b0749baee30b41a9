"""Small scene builders and fixture readers shared by the tests (inputs
only, no method arithmetic)."""
import os

import numpy as np

import nbv_synth as S


def axis_camera(W=64, H=64, f=60.0, z0=0.5):
    """Camera with identity rotation at distance z0 from the origin: a
    Gaussian at world (x, y, z) sits at camera-space (x, y, z + z0)."""
    return S.Cameras(np.eye(3, dtype=np.float32)[None].copy(),
                     np.array([[0.0, 0.0, z0]], np.float32),
                     np.array([f], np.float32), np.array([f], np.float32),
                     np.array([W / 2], np.float32), np.array([H / 2], np.float32),
                     np.array([W], np.int32), np.array([H], np.int32))


def make_scene(means, log_scales, quats=None, opacity=None, sh=None, obj=None, K=1, deg=0):
    n = len(means)
    means = np.asarray(means, np.float32).reshape(n, 3)
    log_scales = np.asarray(log_scales, np.float32).reshape(n, 3)
    quats = (np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None
             else np.asarray(quats, np.float32).reshape(n, 4))
    opacity = np.zeros(n, np.float32) if opacity is None else np.asarray(opacity, np.float32)
    nb = (deg + 1) ** 2
    sh = np.zeros((n, nb, 3), np.float32) if sh is None else np.asarray(sh, np.float32).reshape(n, nb, 3)
    obj = np.zeros((n, K + 1), np.float32) if obj is None else np.asarray(obj, np.float32).reshape(n, K + 1)
    return S.Scene(means, log_scales, quats, opacity, sh, obj, deg, K)


def random_small_scene(seed, n=6, K=2, deg=1, spread=0.05, depth=0.0):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-spread, spread, n), rng.uniform(-spread, spread, n),
                      depth + rng.uniform(-spread, spread, n)], 1)
    log_scales = rng.normal(np.log(0.012), 0.25, (n, 3))
    q = rng.standard_normal((n, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = rng.normal(-0.5, 0.6, n)
    nb = (deg + 1) ** 2
    sh = np.zeros((n, nb, 3)); sh[:, 0, :] = rng.uniform(0.2, 1.5, (n, 3))
    if nb > 1:
        sh[:, 1:, :] = rng.normal(0, 0.1, (n, nb - 1, 3))
    obj = rng.normal(0, 1.0, (n, K + 1))
    return make_scene(means, log_scales, q, opacity, sh, obj, K, deg)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_hyperparameters():
    """{name: value} from golden/paper_hyperparameters.txt (values printed
    in the paper, each line with its citation)."""
    out = {}
    with open(os.path.join(GOLDEN, "paper_hyperparameters.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, cite = line.split(None, 2)
            assert cite.startswith("Sec."), line
            out[name] = float(value)
    return out
