"""Seeded synthetic inputs for the object-aware Gaussian-splat NBV scorer.

This module only *draws* inputs: Gaussian scenes laid out like cluttered
tabletop scenes, and pinhole cameras on a sphere around the scene centre.
It holds none of the method's arithmetic (no projection, compositing,
Jacobians or information gain), so that both the CUDA path and the CPU
oracle can be fed the same arrays without sharing any of the method.

Scene structure follows the paper's evaluation setup (Sec. IV-A.1):
objects cluttered on a table, candidate views on a sphere centred at the
scene centroid that mix random viewpoints with a spiral ring at one
latitude, and a few initial training views (4 initial views, Sec. IV-A.3).

Parameter conventions (the paper's Gaussian parameterisation, Sec. III-A.1):
  means        (N,3)  world-space centres mu, metres, z up, table at z=0
  log_scales   (N,3)  natural log of the per-axis standard deviations s
  quats        (N,4)  rotation r as (w,x,y,z); drawn unit-norm
  opacity      (N,)   opacity logit rho (opacity sigma = sigmoid(rho))
  sh           (N,(d+1)^2,3) spherical-harmonic colour coefficients c
  obj_logits   (N,K+1) object logits o; channel 0 is the background id

Cameras are world->camera rigid transforms in OpenCV axes (x right, y down,
z forward):  x_cam = R @ x_world + t.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene",
    "Cameras",
    "Workload",
    "look_at",
    "sphere_cameras",
    "training_cameras",
    "uniform_cube_scene",
    "tabletop_scene",
    "make_workload",
    "CONFIGS",
]


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    obj_logits: np.ndarray
    sh_degree: int
    K: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity[idx].copy(),
                     self.sh[idx].copy(), self.obj_logits[idx].copy(),
                     self.sh_degree, self.K)


@dataclass
class Cameras:
    R: np.ndarray        # (n,3,3) float32, world->camera rotation, row-major
    t: np.ndarray        # (n,3) float32
    fx: np.ndarray       # (n,) float32
    fy: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    width: np.ndarray    # (n,) int32
    height: np.ndarray   # (n,) int32

    @property
    def n(self) -> int:
        return int(self.R.shape[0])

    def subset(self, idx) -> "Cameras":
        idx = np.atleast_1d(np.asarray(idx))
        return Cameras(self.R[idx].copy(), self.t[idx].copy(), self.fx[idx].copy(),
                       self.fy[idx].copy(), self.cx[idx].copy(), self.cy[idx].copy(),
                       self.width[idx].copy(), self.height[idx].copy())

    @staticmethod
    def concat(parts) -> "Cameras":
        return Cameras(*[np.concatenate([getattr(p, f) for p in parts])
                         for f in ("R", "t", "fx", "fy", "cx", "cy", "width", "height")])


@dataclass
class Workload:
    name: str
    scene: Scene
    train: Cameras
    cand: Cameras
    target: int = -1              # -1: whole scene; otherwise object id (Eq. 12)
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# cameras

def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """World->camera (R, t) for a camera at `position` looking at `target`,
    OpenCV axes (x right, y down, z forward), world up +z."""
    p = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - p
    f /= np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, dtype=np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f], axis=0)
    t = -R @ p
    return R, t


def _cams_from_positions(pos, width, height, focal):
    n = len(pos)
    R = np.zeros((n, 3, 3), np.float32)
    t = np.zeros((n, 3), np.float32)
    for i, p in enumerate(pos):
        Ri, ti = look_at(p)
        R[i], t[i] = Ri, ti
    width = np.broadcast_to(np.asarray(width, np.int32), (n,)).copy()
    height = np.broadcast_to(np.asarray(height, np.int32), (n,)).copy()
    focal = np.broadcast_to(np.asarray(focal, np.float32), (n,)).copy()
    return Cameras(R, t, focal.copy(), focal.copy(),
                   (width.astype(np.float32) * 0.5), (height.astype(np.float32) * 0.5),
                   width, height)


def _sph(r, elev, azim):
    return np.stack([r * np.cos(elev) * np.cos(azim),
                     r * np.cos(elev) * np.sin(azim),
                     r * np.sin(elev)], axis=-1)


def sphere_cameras(rng, n, radius, width, height, focal,
                   ring_elev_deg=45.0, cap_elev_deg=(20.0, 80.0)):
    """Candidate views (Sec. IV-A.1): half on a spiral ring at one latitude,
    evenly spaced in longitude, half uniform (by area) on a spherical cap.
    `radius`, `width`, `height`, `focal` may be scalars or per-view arrays."""
    n_ring = n // 2
    n_cap = n - n_ring
    radius = np.broadcast_to(np.asarray(radius, np.float64), (n,))
    az_ring = np.arange(n_ring) * (2.0 * math.pi / max(n_ring, 1))
    el_ring = np.full(n_ring, math.radians(ring_elev_deg))
    s0, s1 = math.sin(math.radians(cap_elev_deg[0])), math.sin(math.radians(cap_elev_deg[1]))
    el_cap = np.arcsin(rng.uniform(s0, s1, n_cap))
    az_cap = rng.uniform(0.0, 2.0 * math.pi, n_cap)
    el = np.concatenate([el_ring, el_cap])
    az = np.concatenate([az_ring, az_cap])
    pos = _sph(radius, el, az)
    return _cams_from_positions(pos, width, height, focal)


def training_cameras(width, height, focal, radius=0.6, elev_deg=50.0,
                     azim_deg=(0.0, 25.0, 50.0, 75.0)):
    """The initial training views: a few neighbouring poses on one side of
    the scene (4 initial views, Sec. IV-A.3)."""
    az = np.radians(np.asarray(azim_deg, np.float64))
    el = np.full_like(az, math.radians(elev_deg))
    pos = _sph(np.full_like(az, radius), el, az)
    return _cams_from_positions(pos, width, height, focal)


# ----------------------------------------------------------------------------
# Gaussians

def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _random_rotation(rng):
    """A uniformly random 3x3 rotation (QR of a Gaussian matrix, sign-fixed);
    used only to orient the synthetic object blobs."""
    Q, Rr = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(Rr))[None, :]
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def _object_logits(ids, kappa, K):
    """One-hot-like object logits: o[id] = tau, 0 elsewhere, with tau chosen
    so that the largest softmax probability equals
    1/(K+1) + kappa * (1 - 1/(K+1)), capped at 1 - 1e-6."""
    n = ids.shape[0]
    pm = 1.0 / (K + 1) + kappa * (1.0 - 1.0 / (K + 1))
    pm = np.minimum(pm, 1.0 - 1e-6)
    tau = np.log(K * pm / (1.0 - pm))
    o = np.zeros((n, K + 1), np.float64)
    o[np.arange(n), ids] = tau
    return o


def _sh(rng, n, degree):
    nb = (degree + 1) ** 2
    sh = np.zeros((n, nb, 3), np.float64)
    # DC coefficient uniform on +-sqrt(pi): a DC-only colour of U(0,1)
    sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), (n, 3))
    if nb > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, nb - 1, 3))
    return sh


def _kmeans_ids(rng, x, k, iters=20):
    cent = x[rng.choice(x.shape[0], k, replace=False)].copy()
    lab = np.zeros(x.shape[0], np.int64)
    for _ in range(iters):
        d = ((x[:, None, :] - cent[None, :, :]) ** 2).sum(-1)
        lab = d.argmin(1)
        for j in range(k):
            sel = lab == j
            if sel.any():
                cent[j] = x[sel].mean(0)
    return lab


def _pack(means, log_scales, quats, opacity, sh, obj, degree, K):
    f = np.float32
    return Scene(np.ascontiguousarray(means, f), np.ascontiguousarray(log_scales, f),
                 np.ascontiguousarray(quats, f), np.ascontiguousarray(opacity, f),
                 np.ascontiguousarray(sh, f), np.ascontiguousarray(obj, f), degree, K)


def uniform_cube_scene(seed=0, n=2000, K=4, sh_degree=0, side=0.4, conf="uniform"):
    """Means uniform in a cube of side `side` resting on the z=0 table; object
    ids 1..K from k-means on the positions; confidence ~U(0,1)."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-side / 2, side / 2, n),
                      rng.uniform(-side / 2, side / 2, n),
                      rng.uniform(0.0, side, n)], axis=1)
    log_scales = rng.normal(math.log(0.01), 0.3, (n, 3))
    quats = _unit_quats(rng, n)
    opacity = rng.normal(0.0, 1.0, n)
    sh = _sh(rng, n, sh_degree)
    ids = _kmeans_ids(rng, means, K) + 1
    kappa = rng.uniform(0.0, 1.0, n) if conf == "uniform" else rng.beta(2.0, 2.0, n)
    obj = _object_logits(ids, kappa, K)
    return _pack(means, log_scales, quats, opacity, sh, obj, sh_degree, K)


def tabletop_scene(seed=0, n_objects=100_000, n_blobs=16, n_table=20_000, K=16,
                   sh_degree=3, table=(0.8, 0.6), margin=0.05, conf="beta"):
    """Cluttered tabletop: `n_blobs` anisotropic 3D-normal object blobs
    (per-axis sigma ~U(2,5) cm, random rotation, lifted by their vertical
    sigma) on a `table` (metres) plus a flat table layer (object id 0,
    log-scale_z = log 0.002). Blob b gets object id 1 + (b mod K)."""
    rng = np.random.default_rng(seed)
    tx, ty = table[0] / 2, table[1] / 2
    per = np.full(n_blobs, n_objects // n_blobs)
    per[: n_objects - per.sum()] += 1
    means, ids = [], []
    for b in range(n_blobs):
        c = np.array([rng.uniform(-tx + margin, tx - margin),
                      rng.uniform(-ty + margin, ty - margin), 0.0])
        sig = rng.uniform(0.02, 0.05, 3)
        Rb = _random_rotation(rng)
        cov = Rb @ np.diag(sig ** 2) @ Rb.T
        c[2] = math.sqrt(cov[2, 2])
        means.append(rng.multivariate_normal(c, cov, int(per[b])))
        ids.append(np.full(int(per[b]), 1 + (b % K), np.int64))
    n_obj = int(per.sum())
    means_t = np.stack([rng.uniform(-tx, tx, n_table), rng.uniform(-ty, ty, n_table),
                        np.zeros(n_table)], axis=1)
    means = np.concatenate(means + [means_t])
    ids = np.concatenate(ids + [np.zeros(n_table, np.int64)])
    n = n_obj + n_table
    log_scales = rng.normal(math.log(0.01), 0.3, (n, 3))
    log_scales[n_obj:, 2] = math.log(0.002)
    quats = _unit_quats(rng, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_table)
    quats[n_obj:] = np.stack([np.cos(phi / 2), np.zeros(n_table), np.zeros(n_table),
                              np.sin(phi / 2)], axis=1)
    opacity = rng.normal(0.0, 1.0, n)
    sh = _sh(rng, n, sh_degree)
    kappa = rng.uniform(0.0, 1.0, n) if conf == "uniform" else rng.beta(2.0, 2.0, n)
    obj = _object_logits(ids, kappa, K)
    return _pack(means, log_scales, quats, opacity, sh, obj, sh_degree, K)


# ----------------------------------------------------------------------------
# the workloads

CONFIGS = {
    # 2,000 Gaussians in a 0.4 m cube, K=4, SH degree 0, 8 views at 64x48, f=60
    "tiny": dict(kind="cube", n=2000, K=4, d=0, views=8, W=64, H=48, f=60.0, target=-1),
    # 100k Gaussians in 16 blobs + 20k table, K=16, SH degree 3, 64 views at 640x480, f=525
    "scene": dict(kind="table", n_obj=100_000, blobs=16, n_table=20_000, K=16, d=3,
                  views=64, W=640, H=480, f=525.0, target=-1),
    # 300k Gaussians (280k in 32 blobs + 20k table), K=32, 256 views at mixed
    # resolution (half 320x240 f=262.5, half 640x480 f=525), radii U(0.4,0.8),
    # object-centric target id 1
    "batch": dict(kind="table", n_obj=280_000, blobs=32, n_table=20_000, K=32, d=3,
                  views=256, W=640, H=480, f=525.0, mixed=True, target=1),
    # 500k Gaussians (480k + 20k table), K=32, 4 observed views at 640x480
    "diff": dict(kind="table", n_obj=480_000, blobs=32, n_table=20_000, K=32, d=3,
                 views=4, W=640, H=480, f=525.0, target=-1),
    # 1M Gaussians (980k + 20k table), K=64, 1,024 views at 640x480
    "surrogate": dict(kind="table", n_obj=980_000, blobs=64, n_table=20_000, K=64, d=3,
                      views=1024, W=640, H=480, f=525.0, target=-1),
}


def make_workload(name, seed=0, n_views=None, scale=None) -> Workload:
    """Build one of the named workloads. `n_views` overrides the candidate
    count; `scale` (0<scale<=1) shrinks the Gaussian counts for quick tests
    while keeping the structure."""
    cfg = dict(CONFIGS[name])
    rng = np.random.default_rng(seed + 7919)
    nv = cfg["views"] if n_views is None else int(n_views)
    if cfg["kind"] == "cube":
        n = cfg["n"] if scale is None else max(1, int(cfg["n"] * scale))
        scene = uniform_cube_scene(seed, n=n, K=cfg["K"], sh_degree=cfg["d"])
    else:
        s = 1.0 if scale is None else scale
        scene = tabletop_scene(seed, n_objects=max(cfg["blobs"], int(cfg["n_obj"] * s)),
                               n_blobs=cfg["blobs"], n_table=max(1, int(cfg["n_table"] * s)),
                               K=cfg["K"], sh_degree=cfg["d"])
    if cfg.get("mixed"):
        low = (np.arange(nv) % 2) == 0          # alternate so ring and cap both mix
        W = np.where(low, 320, 640)
        H = np.where(low, 240, 480)
        f = np.where(low, 262.5, 525.0)
        radius = rng.uniform(0.4, 0.8, nv)
        cand = sphere_cameras(rng, nv, radius, W, H, f)
    else:
        cand = sphere_cameras(rng, nv, 0.6, cfg["W"], cfg["H"], cfg["f"])
    train = training_cameras(cfg["W"], cfg["H"], cfg["f"])
    return Workload(name, scene, train, cand, cfg["target"], meta=cfg)
