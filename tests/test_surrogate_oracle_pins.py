"""Pins of the surrogate oracle (oracle/surrogate.py) against hand-worked
values and finite differences, on the CPU."""
import types

import math

import numpy as np
import pytest

from helpers import axis_camera, make_scene
from oracle import oracle as O
from oracle import surrogate as SO


def test_bf16_round_to_nearest_even():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 3.0e-3, 65504.0], np.float32)
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, 0.0030059814453125, 65536.0], np.float32)
    np.testing.assert_array_equal(SO.bf16(x), want)


def _cam(f=100.0, W=80, H=80):
    return types.SimpleNamespace(n=1, R=np.eye(3, dtype=np.float32)[None], t=np.array([[0, 0, 1]], np.float32),
                                 fx=np.array([f], np.float32), fy=np.array([f], np.float32),
                                 cx=np.array([W / 2], np.float32), cy=np.array([H / 2], np.float32),
                                 width=np.array([W], np.int32), height=np.array([H], np.int32))


def test_descriptor_hand_worked():
    """Four Gaussians in front of a camera at z = -1 looking along +z: one at
    the image centre (cell (4, 4)), one at pixel (15, 15) (cell (1, 1)), one
    behind the camera and one outside the image (both ignored)."""
    means = np.array([[0, 0, 0], [-0.25, -0.25, 0], [0, 0, -2], [1.0, 0, 0]], np.float32)
    rho = np.array([0.0, np.log(3.0), 0.0, 0.0], np.float32)          # sigma 0.5, 0.75
    K = 3
    logits = np.zeros((4, K + 1), np.float32)
    logits[0, 2] = 5.0
    logits[1, 1] = 5.0
    scene = types.SimpleNamespace(n=4, K=K, means=means, opacity=rho, obj_logits=logits)
    conf = np.array([2.0, 4.0, 7.0, 9.0])
    # a training camera at the candidate's own pose (novelty 0 for every
    # Gaussian) and one on the opposite side (novelty 2 - (1 - cos) ...)
    raw = np.zeros(448)
    raw[36], raw[9] = 0.5, 0.75                                       # sigma
    raw[64 + 36], raw[64 + 9] = 1.0, 3.0                              # c sigma
    raw[128 + 36], raw[128 + 9] = 1.0, 3.0                            # c sigma / z (z = 1)
    raw[192 + 36], raw[192 + 9] = 1.0 / 2.0, 3.0 / 4.0                # c sigma / (1 + o)
    raw[384 + 2], raw[384 + 1] = 1.0, 3.0                             # per object id
    raw[444], raw[445], raw[446], raw[447] = 1.25, 4.0, 1.25, 4.0      # totals: sigma, c sigma, cov, /z
    f = np.arange(448)
    scale = np.where(f < 384, 64 / 4, np.where(f < 440, (K + 1) / 4, 1 / 4))
    d = SO.descriptors(scene, _cam(), conf, obs=np.array([1.0, 3.0, 0.0, 0.0]), train=_cam())[0]
    np.testing.assert_allclose(d, np.log1p(raw * scale), rtol=1e-6, atol=1e-12)
    # novelty: a training camera on the far side of the scene (centre (0, 0, 1)
    # looking along -z) sees the centre Gaussian from the opposite direction
    far = _cam()
    far.R = np.diag([1.0, -1.0, -1.0]).astype(np.float32)[None]
    far.t = np.array([[0, 0, 1]], np.float32)
    d2 = SO.descriptors(scene, _cam(), conf, train=far)[0]
    # Gaussian 0: directions (0,0,1) vs (0,0,-1): nu = 2; Gaussian 1 at
    # (-.25,-.25,0): cosine of (-.25,-.25,1) with (-.25,-.25,-1), nu = 1 - (1/8 - 1)/(1 + 1/8)
    nu1 = 1 - (0.125 - 1) / 1.125
    assert np.expm1(d2[256 + 36]) / 16 == pytest.approx(2.0 * 1.0, rel=1e-6)
    assert np.expm1(d2[256 + 9]) / 16 == pytest.approx(3.0 * nu1, rel=1e-6)
    assert np.expm1(d2[320 + 9]) / 16 == pytest.approx(3.0 * nu1 ** 2, rel=1e-6)


def _params(d_in, width, rng, scale=0.5):
    o = SO.layout(d_in, width)
    return rng.normal(0, scale, o["P"])


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    d_in, width, B = 5, 16, 7
    p = _params(d_in, width, rng)
    x = rng.normal(0, 1, (B, d_in))
    t = rng.normal(0, 1, B)
    g, loss = SO.gradients(p, x, t, d_in, width, rounding=False)
    h = 1e-6
    for i in rng.choice(len(p), 60, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        lp = SO.gradients(p + e, x, t, d_in, width, rounding=False)[1]
        lm = SO.gradients(p - e, x, t, d_in, width, rounding=False)[1]
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-6 * (1 + abs(g[i])), i
    y, _ = SO.forward(p, x, d_in, width, rounding=False)
    assert loss == pytest.approx(np.mean((y - t) ** 2))


def test_mlp_rounding_is_exact_on_representable_values():
    """Small integers are bfloat16 numbers: with integer inputs and weights
    and zero biases the rounded network equals the unrounded one."""
    rng = np.random.default_rng(4)
    d_in, width = 3, 16
    o = SO.layout(d_in, width)
    p = np.zeros(o["P"])
    p[o["W1"]:o["b1"]] = rng.integers(-1, 2, width * d_in)
    p[o["W2"]:o["b2"]] = rng.integers(-1, 2, width * width)
    p[o["w3"]:o["b3"]] = rng.integers(-2, 3, width)
    x = rng.integers(0, 3, (9, d_in)).astype(np.float64)
    y1, _ = SO.forward(p, x, d_in, width, rounding=True)
    y0, _ = SO.forward(p, x, d_in, width, rounding=False)
    np.testing.assert_array_equal(y1, y0)
    W1 = p[o["W1"]:o["b1"]].reshape(width, d_in)
    W2 = p[o["W2"]:o["b2"]].reshape(width, width)
    w3 = p[o["w3"]:o["b3"]]
    np.testing.assert_array_equal(y0, np.maximum(np.maximum(x @ W1.T, 0) @ W2.T, 0) @ w3)


def test_view_w2_single_isotropic_splat():
    """One isotropic splat on the optical axis: T = 1 at every pixel, so the
    per-Gaussian sum of w^2 is the sum of alpha^2 ~ integral pi s2^2
    (sigma^2 - 1/255^2) of the truncated squared Gaussian (s2^2 = (f s/z)^2
    + 0.3), within the jump at the cut-off circle."""
    s, sigma, z0, f = 0.05, 0.3, 0.5, 60.0
    rho = math.log(sigma / (1 - sigma))
    sc = make_scene([[0, 0, 0]], [[math.log(s)] * 3], opacity=[rho], obj=[[0.0, 1.0]], K=1)
    cam = axis_camera(64, 64, f, z0)
    w2 = O.OracleScene(sc).view_w2(cam, 0)
    sig32 = float(np.float32(1.0 / (1.0 + math.exp(-rho))))
    s2sq = (f * float(np.float32(s)) / z0) ** 2 + float(np.float32(0.3))
    integral = math.pi * s2sq * (sig32 ** 2 - 1 / 255 ** 2)
    r_c = math.sqrt(s2sq) * math.sqrt(2 * math.log(255 * sig32))
    edge = 2 * math.pi * r_c / 255 ** 2
    assert abs(w2[0] - integral) < edge
    a = O.OracleScene(sc).render(cam, 0)["alpha"]
    assert w2[0] == pytest.approx(float((a ** 2).sum()), rel=1e-12)
