"""Python front of the CPU oracle (nbv_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers. The product path never
imports this module.

`build()` compiles the oracle with g++ (double precision, no fast-math, no
floating-point contraction, OpenMP). `OracleScene` wraps one Gaussian scene.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbv_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libnbv_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int
    lib.orc_scene_create.restype = P
    lib.orc_scene_create.argtypes = [i64, i32, i32] + [P] * 6 + [P, i32]
    lib.orc_scene_destroy.argtypes = [P]
    lib.orc_confidence.argtypes = [P, P]
    lib.orc_project32.argtypes = [P, P, P, P, P, P, P, P]
    lib.orc_project64.argtypes = [P, P, P, P]
    lib.orc_view_w2.restype = None
    lib.orc_view_w2.argtypes = [P, P, P, P]
    lib.orc_tile_lists.restype = i64
    lib.orc_tile_lists.argtypes = [P, P, P, P, P, i64]
    lib.orc_tile_needed.restype = i64
    lib.orc_tile_needed.argtypes = [P, P, P, P, P, i64]
    lib.orc_render.argtypes = [P, P, P, P, P, P, P, P, P]
    lib.orc_view_blocks.argtypes = [P, P, P, P, P, P, P]
    lib.orc_score.restype = i32
    lib.orc_score.argtypes = [P, i32, P, P, i32, P, P, P, P, P, P, i32]
    lib.orc_sh_basis.argtypes = [i32, i64, P, P]
    lib.orc_prepare.restype = i32
    lib.orc_prepare.argtypes = [P, i32, P, P, i32]
    lib.orc_score_views.restype = i32
    lib.orc_score_views.argtypes = [P, i32, P, P, P, i32]
    lib.orc_freeze.restype = P
    lib.orc_freeze.argtypes = [P, P, P]
    lib.orc_frozen_destroy.argtypes = [P]
    lib.orc_render_frozen.argtypes = [P, P, P, P, P, P, P, P]
    lib.orc_num_threads.restype = i32
    _lib = lib
    return lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


@dataclass
class Hyper:
    """Hyper-parameters of the score (Sec. IV-A.2) and the rasterizer
    conventions the oracle follows."""
    alpha_obj: float = 0.3
    alpha_opa: float = 0.3
    beta_d: float = 10.0
    beta_o: float = 1.0
    lam: float = 0.1
    near: float = 0.2
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    dilation: float = 0.3
    guard: float = 1.3
    tile_w: int = 16
    tile_h: int = 16
    crit: int = 0          # 0 log det (Eq. 6), 1 tr(H_T^-1 c A), 2 tr(c A)

    def array(self):
        return np.array([self.alpha_obj, self.alpha_opa, self.beta_d, self.beta_o, self.lam,
                         self.near, self.alpha_min, self.alpha_max, self.t_min, self.dilation,
                         self.guard, self.tile_w, self.tile_h, self.crit], np.float32)


def cam_arrays(cams, i):
    """(16 floats: R row-major, t, fx, fy, cx, cy), (W, H) of camera i."""
    c = np.concatenate([cams.R[i].reshape(9), cams.t[i].reshape(3),
                        [cams.fx[i], cams.fy[i], cams.cx[i], cams.cy[i]]]).astype(np.float32)
    wh = np.array([cams.width[i], cams.height[i]], np.int32)
    return np.ascontiguousarray(c), wh


def all_cam_arrays(cams):
    cs, whs = zip(*[cam_arrays(cams, i) for i in range(cams.n)]) if cams.n else ((), ())
    c = np.ascontiguousarray(np.stack(cs)) if cams.n else np.zeros((0, 16), np.float32)
    wh = np.ascontiguousarray(np.stack(whs)) if cams.n else np.zeros((0, 2), np.int32)
    return c, wh


def num_threads() -> int:
    return int(_load().orc_num_threads())


def sh_basis(degree: int, dirs: np.ndarray) -> np.ndarray:
    """Real spherical harmonics up to `degree` at unit directions (n,3)."""
    lib = _load()
    dirs = np.ascontiguousarray(dirs, np.float64)
    n = dirs.shape[0]
    Y = np.zeros((n, (degree + 1) ** 2), np.float64)
    lib.orc_sh_basis(degree, n, _ptr(dirs), _ptr(Y))
    return Y


class _Frozen:
    def __init__(self, lib, h):
        self.lib, self.h = lib, h

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_frozen_destroy(self.h)
            self.h = None


class OracleScene:
    """One Gaussian scene held by the oracle."""

    def __init__(self, scene, hyper: Hyper | None = None, target: int = -1):
        self.lib = _load()
        self.hyper = hyper or Hyper()
        self.n, self.K, self.deg = scene.n, scene.K, scene.sh_degree
        self.nb = (self.deg + 1) ** 2
        self._keep = [np.ascontiguousarray(a, np.float32) for a in
                      (scene.means, scene.log_scales, scene.quats, scene.opacity,
                       scene.sh, scene.obj_logits)]
        hp = self.hyper.array()
        self._h = self.lib.orc_scene_create(self.n, self.K, self.deg,
                                            *[_ptr(a) for a in self._keep], _ptr(hp), int(target))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.orc_scene_destroy(h)
            self._h = None

    # parameter counts per output: rgb, depth, objects
    @property
    def lsizes(self):
        return 11 + 3 * self.nb, 11, 12 + self.K

    def confidence(self):
        c = np.zeros(self.n, np.float64)
        self.lib.orc_confidence(self._h, _ptr(c))
        return c

    def view_w2(self, cams, i):
        """Per Gaussian, sum over view i's pixels of (alpha T)^2."""
        c, wh = cam_arrays(cams, i)
        w2 = np.zeros(self.n, np.float64)
        self.lib.orc_view_w2(self._h, _ptr(c), _ptr(wh), _ptr(w2))
        return w2

    def project32(self, cams, i):
        c, wh = cam_arrays(cams, i)
        n = self.n
        rect = np.zeros((n, 4), np.int32)
        radius = np.zeros(n, np.float32)
        zbits = np.zeros(n, np.uint32)
        m2 = np.zeros((n, 2), np.float32)
        conic = np.zeros((n, 3), np.float32)
        self.lib.orc_project32(self._h, _ptr(c), _ptr(wh), _ptr(rect), _ptr(radius),
                               _ptr(zbits), _ptr(m2), _ptr(conic))
        return dict(rect=rect, radius=radius, zbits=zbits, mean2d=m2, conic=conic)

    def project64(self, cams, i):
        c, wh = cam_arrays(cams, i)
        v = np.zeros((self.n, 10), np.float64)
        self.lib.orc_project64(self._h, _ptr(c), _ptr(wh), _ptr(v))
        return v

    def _lists(self, fn, cams, i):
        c, wh = cam_arrays(cams, i)
        tw, th = self.hyper.tile_w, self.hyper.tile_h
        nt = ((int(wh[0]) + tw - 1) // tw) * ((int(wh[1]) + th - 1) // th)
        off = np.zeros(nt + 1, np.int64)
        tot = fn(self._h, _ptr(c), _ptr(wh), _ptr(off), None, 0)
        ids = np.zeros(max(tot, 1), np.int32)
        fn(self._h, _ptr(c), _ptr(wh), _ptr(off), _ptr(ids), tot)
        return off, ids[:tot]

    def tile_lists(self, cams, i):
        """Per-tile lists of view i: every splat whose 3-sigma rectangle
        covers the tile, in (depth bits, index) order (offsets, ids)."""
        return self._lists(self.lib.orc_tile_lists, cams, i)

    def tile_needed(self, cams, i):
        """The entries of tile_lists that pass the skip test (1/255 cut-off,
        power <= 0) at some in-image pixel centre of their tile: those no
        valid list may drop (offsets, ids, same order)."""
        return self._lists(self.lib.orc_tile_needed, cams, i)

    def render(self, cams, i):
        c, wh = cam_arrays(cams, i)
        W, H = int(wh[0]), int(wh[1])
        KC = self.K + 1
        rgb = np.zeros((H, W, 3)); depth = np.zeros((H, W)); alpha = np.zeros((H, W))
        obj = np.zeros((H, W, KC)); nc = np.zeros((H, W), np.int32)
        margin = np.zeros((H, W), np.float32)
        self.lib.orc_render(self._h, _ptr(c), _ptr(wh), _ptr(rgb), _ptr(depth), _ptr(alpha),
                            _ptr(obj), _ptr(nc), _ptr(margin))
        return dict(rgb=rgb, depth=depth, alpha=alpha, obj=obj, n_contrib=nc, margin=margin)

    def freeze(self, cams, i):
        """Record this scene's discrete compositing decisions in view i."""
        c, wh = cam_arrays(cams, i)
        return _Frozen(self.lib, self.lib.orc_freeze(self._h, _ptr(c), _ptr(wh)))

    def render_frozen(self, frozen, cams, i):
        """Render view i of this scene with the decisions recorded in `frozen`."""
        c, wh = cam_arrays(cams, i)
        W, H = int(wh[0]), int(wh[1])
        rgb = np.zeros((H, W, 3)); depth = np.zeros((H, W)); alpha = np.zeros((H, W))
        obj = np.zeros((H, W, self.K + 1))
        self.lib.orc_render_frozen(self._h, frozen.h, _ptr(c), _ptr(wh), _ptr(rgb), _ptr(depth),
                                   _ptr(alpha), _ptr(obj))
        return dict(rgb=rgb, depth=depth, alpha=alpha, obj=obj)

    def view_blocks(self, cams, i, mask=None):
        """Dense Jacobian blocks A^f_g (Eqs. 6, 9) of one view for the
        Gaussians selected by `mask` (all if None), in index order."""
        c, wh = cam_arrays(cams, i)
        m = self.n if mask is None else int(np.count_nonzero(mask))
        lr, ld, lo = self.lsizes
        Ar = np.zeros((m, lr, lr)); Ad = np.zeros((m, ld, ld)); Ao = np.zeros((m, lo, lo))
        mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
        self.lib.orc_view_blocks(self._h, _ptr(c), _ptr(wh), _ptr(mk), _ptr(Ar), _ptr(Ad), _ptr(Ao))
        return Ar, Ad, Ao

    def prepare(self, train, row_stride: int = 1):
        """Keep the training state H_T (Eqs. 6, 9) for score_views()."""
        tc, twh = all_cam_arrays(train)
        rc = self.lib.orc_prepare(self._h, train.n, _ptr(tc), _ptr(twh), int(row_stride))
        if rc != 0:
            raise RuntimeError(f"orc_prepare failed: {rc}")

    def score_views(self, cams, row_stride: int = 1):
        """Raw gains IG_f of each view against the kept training state."""
        cc, cwh = all_cam_arrays(cams)
        ig = np.zeros((cams.n, 3))
        rc = self.lib.orc_score_views(self._h, cams.n, _ptr(cc), _ptr(cwh), _ptr(ig), int(row_stride))
        if rc != 0:
            raise RuntimeError(f"orc_score_views failed: {rc}")
        return ig

    def score(self, train, cand, delta_view: int = -1):
        """IG of every training view and candidate (Eqs. 5-11 or 12), the
        normalised weighted score and the NBV argmax."""
        tc, twh = all_cam_arrays(train)
        cc, cwh = all_cam_arrays(cand)
        igt = np.zeros((train.n, 3)); igc = np.zeros((cand.n, 3)); sc = np.zeros(cand.n)
        delta = np.zeros((self.n, 3)) if delta_view >= 0 else None
        best = self.lib.orc_score(self._h, train.n, _ptr(tc), _ptr(twh), cand.n, _ptr(cc),
                                  _ptr(cwh), _ptr(igt), _ptr(igc), _ptr(sc), _ptr(delta),
                                  int(delta_view))
        return dict(ig_train=igt, ig_cand=igc, score=sc, best=int(best), delta=delta)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
