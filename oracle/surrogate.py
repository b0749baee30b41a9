"""CPU oracle of the learned candidate pre-scoring: the per-view descriptor
and the 3-layer MLP (forward pass and the gradient of its mean squared
error), written out plainly in double precision.

TEST INFRASTRUCTURE ONLY: the test-suite is the only caller. The product
path never imports this module.

Descriptor: for every Gaussian whose centre projects in front of the near
plane and inside the image, with opacity sigma, confidence c (Eq. 7 / 12),
camera depth z, training observation o (sum over the training views'
pixels of w^2, w = alpha T) and angular novelty nu (1 - the largest cosine
between the direction from the candidate's centre to the Gaussian and the
directions from the training cameras' centres), sums over an 8 x 8 grid of
image cells of sigma, c sigma, c sigma / z, c sigma / (1 + o), c sigma nu,
c sigma nu^2; sums of c sigma per most probable object id (56 bins, larger
ids in the last); view totals of c sigma nu, c sigma [nu > 0.1],
c sigma [nu > 0.3], c sigma sqrt(nu), sigma, c sigma, c sigma / (1 + o),
c sigma / z; then log(1 + s x) with s = 64 / n (cells), (K + 1) / n
(objects) or 1 / n (totals). The centre,
the cell and the in-image test are the discrete decisions; they are taken
in single precision in one fixed order of correctly rounded operations
(numpy float32 arithmetic, no fused multiply-add), the sums in double.

MLP: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3 with the
input, W1, W2 and the hidden activations rounded to bfloat16 (round to
nearest even), everything else in double; the gradient of
mean_m (y_m - t_m)^2 is the chain rule through that function (the roundings
pass gradients through unchanged).
"""
from __future__ import annotations

import numpy as np

DESC_DIM = 448


def bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), kept in float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _centres(cams):
    """Camera centres -R^T t (double)."""
    R = np.asarray(cams.R, np.float64).reshape(cams.n, 3, 3)
    t = np.asarray(cams.t, np.float64).reshape(cams.n, 3)
    return -np.einsum("nji,nj->ni", R, t)


def descriptors(scene, cams, conf, obs=None, train=None, near=0.2):
    """[n_views, 448] descriptors (see the module docstring). conf: c_g per
    Gaussian (float64), as the oracle's confidence gives it; obs: the
    training observation per Gaussian (zero when None); train: the training
    cameras (novelty 1 when None)."""
    f32 = np.float32
    n, K = scene.n, scene.K
    mu = np.asarray(scene.means, f32)
    mu64 = mu.astype(np.float64)
    sig = (1.0 / (1.0 + np.exp(-np.asarray(scene.opacity, np.float64).reshape(n)))).astype(f32)
    c = np.asarray(conf, np.float64).astype(f32)
    logits = np.asarray(scene.obj_logits, np.float64).reshape(n, K + 1)
    ids = np.minimum(np.argmax(logits, axis=1), 55)          # lowest id on ties
    cs = (c * sig).astype(f32).astype(np.float64)
    o = np.zeros(n) if obs is None else np.asarray(obs, np.float64)
    cov = cs / (1.0 + o)
    if train is not None:
        dt = mu64[None] - _centres(train).astype(np.float32).astype(np.float64)[:, None]
        dt /= np.linalg.norm(dt, axis=2, keepdims=True)
    cv = _centres(cams).astype(np.float32).astype(np.float64)
    out = np.zeros((cams.n, DESC_DIM), np.float64)
    for v in range(cams.n):
        R = np.asarray(cams.R[v], f32).reshape(3, 3)
        t = np.asarray(cams.t[v], f32).reshape(3)
        fx, fy, cx, cy = (f32(cams.fx[v]), f32(cams.fy[v]), f32(cams.cx[v]), f32(cams.cy[v]))
        W, H = f32(cams.width[v]), f32(cams.height[v])
        tc = []
        for r in range(3):
            a = (R[r, 0] * mu[:, 0] + R[r, 1] * mu[:, 1]).astype(f32)
            a = (a + R[r, 2] * mu[:, 2]).astype(f32)
            tc.append((a + t[r]).astype(f32))
        tx, ty, tz = tc
        front = tz > f32(near)
        tzs = np.where(front, tz, f32(1.0))
        mx = (fx * (tx / tzs).astype(f32)).astype(f32) + cx
        my = (fy * (ty / tzs).astype(f32)).astype(f32) + cy
        ok = front & (mx >= 0) & (mx < W) & (my >= 0) & (my < H)
        ix = np.minimum(7, np.floor(((f32(8.0) * mx).astype(f32) / W).astype(f32))).astype(np.int64)
        iy = np.minimum(7, np.floor(((f32(8.0) * my).astype(f32) / H).astype(f32))).astype(np.int64)
        cell = (iy * 8 + ix)[ok]
        if train is not None:
            d = mu64 - cv[v]
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            nu = np.maximum(0.0, 1.0 - np.max(np.einsum("tnk,nk->tn", dt, d), axis=0))
        else:
            nu = np.ones(n)
        csz = (cs.astype(f32) / tz).astype(f32).astype(np.float64)
        h = np.zeros(DESC_DIM, np.float64)
        w = [sig.astype(np.float64), cs, csz, cov, cs * nu, cs * nu * nu]
        for b, wb in enumerate(w):
            np.add.at(h, 64 * b + cell, wb[ok])
        np.add.at(h, 384 + ids[ok], cs[ok])
        tot = [cs * nu, cs * (nu > 0.1), cs * (nu > 0.3), cs * np.sqrt(nu), sig.astype(np.float64), cs, cov, csz]
        for b, wb in enumerate(tot):
            h[440 + b] = wb[ok].sum()
        f = np.arange(DESC_DIM)
        scale = np.where(f < 384, 64.0 / n, np.where(f < 440, (K + 1) / n, 1.0 / n))
        out[v] = np.log1p(h * scale)
    return out


def layout(d_in, width):
    """Offsets of W1, b1, W2, b2, w3, b3 in the flattened parameters."""
    o = {}
    o["W1"] = 0
    o["b1"] = o["W1"] + width * d_in
    o["W2"] = o["b1"] + width
    o["b2"] = o["W2"] + width * width
    o["w3"] = o["b2"] + width
    o["b3"] = o["w3"] + width
    o["P"] = o["b3"] + 1
    return o


def unpack(params, d_in, width):
    o = layout(d_in, width)
    p = np.asarray(params, np.float64)
    return (p[o["W1"]:o["b1"]].reshape(width, d_in), p[o["b1"]:o["W2"]], p[o["W2"]:o["b2"]].reshape(width, width),
            p[o["b2"]:o["w3"]], p[o["w3"]:o["b3"]], p[o["b3"]])


def forward(params, x, d_in, width, rounding=True):
    """y [B] and the intermediates; rounding=False skips the bfloat16
    roundings (a plain double-precision network, used to pin the gradient)."""
    W1, b1, W2, b2, w3, b3 = unpack(params, d_in, width)
    rnd = (lambda a: bf16(np.asarray(a, np.float32)).astype(np.float64)) if rounding else \
        (lambda a: np.asarray(a, np.float64))
    X = rnd(x)
    W1b, W2b = rnd(W1), rnd(W2)
    a1 = X @ W1b.T + b1.astype(np.float64)
    h1 = rnd(np.maximum(a1, 0.0))
    a2 = h1 @ W2b.T + b2.astype(np.float64)
    h2 = rnd(np.maximum(a2, 0.0))
    y = h2 @ w3.astype(np.float64) + float(b3)
    return y, dict(X=X, W1b=W1b, W2b=W2b, h1=h1, h2=h2)


def gradients(params, x, t, d_in, width, rounding=True):
    """(flattened gradient in the parameter order, loss)."""
    W1, b1, W2, b2, w3, b3 = unpack(params, d_in, width)
    y, c = forward(params, x, d_in, width, rounding)
    B = len(y)
    r = y - np.asarray(t, np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    dw3 = c["h2"].T @ dy
    db3 = dy.sum()
    dz2 = np.outer(dy, w3.astype(np.float64)) * (c["h2"] > 0)
    dW2 = dz2.T @ c["h1"]
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ c["W2b"]
    dz1 = dh1 * (c["h1"] > 0)
    dW1 = dz1.T @ c["X"]
    db1 = dz1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return g, loss
