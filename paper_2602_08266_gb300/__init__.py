"""GB300 object-aware Gaussian-splat next-best-view scorer (arXiv 2602.08266).

A thin Python binding over the C ABI of include/nbvgs.h (libnbvgs.so, built
in-tree by `build()`); it only marshals arguments. Every step of the
rendering and scoring runs in the library's CUDA kernels; there is no CPU
fallback: if the library is missing, `NBVScorer` raises.

Typical use (PyTorch is used for device memory and the current stream):

    sc = NBVScorer(K=16, sh_degree=3)
    sc.load_gaussians(means, log_scales, quats, opacity, sh, obj_logits)
    sc.set_train_views(train_cams); sc.set_candidates(cand_cams)
    sc.prepare(target=-1)                 # -1: whole scene (Eq. 7); k: object k (Eq. 12)
    ig = sc.score()                       # [n_cand, 4]: IG_rgb, IG_d, IG_o, weighted total
    best, best_score = sc.argmax()        # the next best view (Eq. 5)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["NBVScorer", "NBVError", "build", "load_library", "config_default", "LIB_PATH"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnbvgs.so")

NBV_OK = 0
ERRORS = {-1: "NBV_ERR_ARG", -2: "NBV_ERR_CUDA", -3: "NBV_ERR_OOM", -4: "NBV_ERR_STATE",
          -5: "NBV_ERR_TIMEOUT", -6: "NBV_ERR_EMPTY", -7: "NBV_ERR_UNIMPLEMENTED"}


class NBVError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class nbv_config(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("sh_degree", ctypes.c_int),
                ("alpha_obj", ctypes.c_float), ("alpha_opa", ctypes.c_float),
                ("beta_d", ctypes.c_float), ("beta_o", ctypes.c_float),
                ("lambda_damp", ctypes.c_float), ("near_z", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("t_min", ctypes.c_float), ("dilation", ctypes.c_float), ("guard", ctypes.c_float),
                ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("batched", ctypes.c_int),
                ("stage", ctypes.c_int), ("max_batch_views", ctypes.c_int), ("criterion", ctypes.c_int),
                ("tf32_contraction", ctypes.c_int)]


class nbv_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int)]


_lib = None

# (name, restype, argtypes) of every entry point declared in include/nbvgs.h
_P = ctypes.c_void_p
_SIGS = [
    ("nbv_config_default", None, [ctypes.POINTER(nbv_config), ctypes.c_int, ctypes.c_int]),
    ("nbv_create", ctypes.c_int, [ctypes.POINTER(nbv_config), _P, ctypes.POINTER(_P)]),
    ("nbv_destroy", None, [_P]),
    ("nbv_load_gaussians", ctypes.c_int, [_P, ctypes.c_int64] + [_P] * 6 + [ctypes.c_int]),
    ("nbv_set_train_views", ctypes.c_int, [_P, ctypes.c_int, _P]),
    ("nbv_set_candidates", ctypes.c_int, [_P, ctypes.c_int, _P]),
    ("nbv_prepare", ctypes.c_int, [_P, ctypes.c_int]),
    ("nbv_render", ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    ("nbv_score", ctypes.c_int, [_P, _P, ctypes.c_int]),
    ("nbv_argmax", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    ("nbv_train_gains", ctypes.c_int, [_P, _P]),
    ("nbv_gaussian_gains", ctypes.c_int, [_P, ctypes.c_int, _P]),
    ("nbv_debug_project", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]),
    ("nbv_debug_tile_lists", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int64,
                                            ctypes.POINTER(ctypes.c_int64)]),
    ("nbv_set_profiling", ctypes.c_int, [_P, ctypes.c_int]),
    ("nbv_phase_times", ctypes.c_int, [_P, _P, _P]),
    ("nbv_work_stats", ctypes.c_int, [_P, ctypes.c_int, _P]),
    ("nbv_measure_fp32_fma", ctypes.c_int, [ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    ("nbv_autotune", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]),
    ("nbv_get_tiling", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    ("nbv_sort_tile_keys_noalloc", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int, _P, _P, _P]),
    ("nbv_render_view", ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    ("nbv_render_backward", ctypes.c_int, [_P, _P] + [_P] * 10),
    ("nbv_descriptors", ctypes.c_int, [_P, _P]),
    ("nbv_mlp_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _P, ctypes.POINTER(_P)]),
    ("nbv_mlp_destroy", None, [_P]),
    ("nbv_mlp_num_params", ctypes.c_int64, [_P]),
    ("nbv_mlp_get_params", ctypes.c_int, [_P, _P]),
    ("nbv_mlp_set_params", ctypes.c_int, [_P, _P]),
    ("nbv_mlp_forward", ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    ("nbv_mlp_gradients", ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    ("nbv_mlp_train_step", ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_float,
                                          ctypes.POINTER(ctypes.c_double)]),
    ("nbv_gemm_bf16", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int64, _P,
                                     ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
    ("nbv_score_pruned", ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_float)]),
    ("nbv_set_entry_limit", ctypes.c_int, [_P, ctypes.c_int64]),
    ("nbv_set_gemm_wait_polls", ctypes.c_int, [ctypes.c_int64]),
    ("nbv_last_error", ctypes.c_char_p, [_P]),
    ("nbv_launch_count", ctypes.c_int64, [_P]),
]


def build(force: bool = False, verbose: bool = False) -> str:
    from . import builder
    return builder.build(force=force, verbose=verbose)


def load_library(path: str = LIB_PATH):
    """Load libnbvgs.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2602_08266_gb300.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return [s[0] for s in _SIGS]


def config_default(K: int, sh_degree: int, **overrides) -> nbv_config:
    lib = load_library()
    cfg = nbv_config()
    lib.nbv_config_default(ctypes.byref(cfg), int(K), int(sh_degree))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def _cams_struct(cams):
    """ctypes array of nbv_camera from an object with arrays R (n,3,3), t,
    fx, fy, cx, cy, width, height (e.g. nbv_synth.Cameras)."""
    n = int(np.asarray(cams.R).shape[0])
    arr = (nbv_camera * max(n, 1))()
    R = np.asarray(cams.R, np.float32).reshape(n, 9)
    t = np.asarray(cams.t, np.float32).reshape(n, 3)
    for i in range(n):
        c = arr[i]
        c.R[:] = R[i].tolist()
        c.t[:] = t[i].tolist()
        c.fx, c.fy = float(cams.fx[i]), float(cams.fy[i])
        c.cx, c.cy = float(cams.cx[i]), float(cams.cy[i])
        c.width, c.height = int(cams.width[i]), int(cams.height[i])
    return n, arr


NOALLOC_MAX_PAIRS = 1 << 20


def measure_fp32_fma(packed: bool = False, stream=None) -> float:
    """FP32 fused multiply-add throughput of the current device in TFLOP/s
    (nbv_measure_fp32_fma): the roofline denominator of the compositing
    kernel, measured rather than derived."""
    import torch
    lib = load_library()
    st = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double(0.0)
    rc = lib.nbv_measure_fp32_fma(1 if packed else 0, ctypes.c_void_p(st.cuda_stream), ctypes.byref(out))
    if rc != NBV_OK:
        raise NBVError(rc, "nbv_measure_fp32_fma failed")
    return float(out.value)


def sort_tile_keys_noalloc(keys_in, vals_in, key_bits, keys_out, vals_out, stream=None):
    """Stable sort of (int64 key, int32 value) device tensors by the low
    key_bits bits into caller-owned outputs, without any device allocation
    (see nbv_sort_tile_keys_noalloc in include/nbvgs.h)."""
    import torch
    lib = load_library()
    n = int(keys_in.numel())
    want = ((keys_in, torch.int64), (vals_in, torch.int32), (keys_out, torch.int64), (vals_out, torch.int32))
    dev = torch.cuda.current_device()
    for t, dt in want:
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_contiguous() or t.numel() != n:
            raise NBVError(-1, "sort_tile_keys_noalloc: keys int64 and values int32, contiguous, all of one length")
        if not t.is_cuda or t.device.index != dev:
            raise NBVError(-1, "sort_tile_keys_noalloc: every tensor must be on the current CUDA device")
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.nbv_sort_tile_keys_noalloc(ctypes.c_void_p(keys_in.data_ptr()),
                                        ctypes.c_void_p(vals_in.data_ptr()), int(keys_in.numel()),
                                        int(key_bits), ctypes.c_void_p(keys_out.data_ptr()),
                                        ctypes.c_void_p(vals_out.data_ptr()),
                                        ctypes.c_void_p(st.cuda_stream))
    if rc != NBV_OK:
        raise NBVError(rc, "nbv_sort_tile_keys_noalloc failed")


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class NBVScorer:
    """One scoring context (nbv_ctx) on the current CUDA device and stream."""

    def __init__(self, K: int, sh_degree: int, stream=None, **overrides):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.cfg = config_default(K, sh_degree, **overrides)
        self.K, self.deg = int(K), int(sh_degree)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.nbv_create(ctypes.byref(self.cfg), ctypes.c_void_p(stream.cuda_stream),
                                 ctypes.byref(h))
        if rc != NBV_OK:
            raise NBVError(rc, "nbv_create failed")
        self._h = h
        self.n = 0
        self.n_train = 0
        self.n_cand = 0
        self._cand = None

    def close(self):
        if getattr(self, "_h", None):
            self.lib.nbv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != NBV_OK:
            msg = self.lib.nbv_last_error(self._h)
            raise NBVError(rc, msg.decode() if msg else "")

    # ---------------------------------------------------------------- inputs
    def load_gaussians(self, means, log_scales, quats, opacity, sh, obj_logits):
        """Copy n Gaussians in. torch CUDA tensors are copied on the device;
        numpy arrays (or CPU tensors) are copied from the host."""
        arrs = [means, log_scales, quats, opacity, sh, obj_logits]
        on_dev = all(hasattr(a, "is_cuda") and a.is_cuda for a in arrs)
        if on_dev:
            keep = [a.detach().float().contiguous() for a in arrs]
            ptrs = [ctypes.c_void_p(a.data_ptr()) for a in keep]
        else:
            keep = [np.ascontiguousarray(a.cpu().numpy() if hasattr(a, "cpu") else a, np.float32)
                    for a in arrs]
            ptrs = [ctypes.c_void_p(a.ctypes.data) for a in keep]
        n = int(keep[0].shape[0])
        self._check(self.lib.nbv_load_gaussians(self._h, n, *ptrs, 1 if on_dev else 0))
        self.n = n
        self._keep = keep

    def load_scene(self, scene):
        """Load an object with the six parameter arrays (e.g. nbv_synth.Scene)."""
        self.load_gaussians(scene.means, scene.log_scales, scene.quats, scene.opacity, scene.sh,
                            scene.obj_logits)

    def set_train_views(self, cams):
        n, arr = _cams_struct(cams)
        self._check(self.lib.nbv_set_train_views(self._h, n, arr))
        self.n_train = n
        self._train = (np.asarray(cams.width).copy(), np.asarray(cams.height).copy())

    def set_candidates(self, cams):
        n, arr = _cams_struct(cams)
        self._check(self.lib.nbv_set_candidates(self._h, n, arr))
        self.n_cand = n
        self._cand = (np.asarray(cams.width).copy(), np.asarray(cams.height).copy())

    # --------------------------------------------------------------- compute
    def prepare(self, target: int = -1):
        self._check(self.lib.nbv_prepare(self._h, int(target)))

    def render(self, cand: int, rgb=True, depth=True, alpha=True, obj=True):
        torch = self.torch
        W, H = int(self._cand[0][cand]), int(self._cand[1][cand])
        dev = torch.device("cuda")
        out = {}
        out["rgb"] = torch.empty((H, W, 3), device=dev) if rgb else None
        out["depth"] = torch.empty((H, W), device=dev) if depth else None
        out["alpha"] = torch.empty((H, W), device=dev) if alpha else None
        out["obj"] = torch.empty((H, W, self.K + 1), device=dev) if obj else None
        self._check(self.lib.nbv_render(self._h, int(cand), _dptr(out["rgb"]), _dptr(out["depth"]),
                                        _dptr(out["alpha"]), _dptr(out["obj"])))
        return {k: v for k, v in out.items() if v is not None}

    def render_camera(self, cams, i: int):
        """Render camera i of `cams` (any camera set): dict of device tensors."""
        torch = self.torch
        _, arr = _cams_struct(cams)
        W, H = int(cams.width[i]), int(cams.height[i])
        dev = torch.device("cuda")
        out = dict(rgb=torch.empty((H, W, 3), device=dev), depth=torch.empty((H, W), device=dev),
                   alpha=torch.empty((H, W), device=dev), obj=torch.empty((H, W, self.K + 1), device=dev))
        self._check(self.lib.nbv_render_view(self._h, ctypes.byref(arr[i]), _dptr(out["rgb"]), _dptr(out["depth"]),
                                             _dptr(out["alpha"]), _dptr(out["obj"])))
        return out

    def render_backward(self, cams, i: int, g_rgb=None, g_depth=None, g_alpha=None, g_obj=None, grads=None):
        """Add the gradients of the loaded Gaussians' raw parameters for the
        given output gradients of camera i (device tensors, any may be None)
        to `grads` (created zero when None); returns grads."""
        torch = self.torch
        n, nb, KC = self.n, (self.deg + 1) ** 2, self.K + 1
        if grads is None:
            z = lambda *s: torch.zeros(s, device="cuda")
            grads = dict(means=z(n, 3), log_scales=z(n, 3), quats=z(n, 4), opacity=z(n), sh=z(n, nb, 3),
                         obj_logits=z(n, KC))
        _, arr = _cams_struct(cams)
        c = lambda t: None if t is None else t.detach().float().contiguous()
        keep = [c(g_rgb), c(g_depth), c(g_alpha), c(g_obj)]
        self._check(self.lib.nbv_render_backward(
            self._h, ctypes.byref(arr[i]), *[_dptr(t) for t in keep],
            *[_dptr(grads[k]) for k in ("means", "log_scales", "quats", "opacity", "sh", "obj_logits")]))
        return grads

    def score(self, out=None):
        """[n_cand, 4] device tensor: IG_rgb, IG_d, IG_o (Eq. 5 per output)
        and the normalised weighted total (Eqs. 10-11)."""
        torch = self.torch
        if out is None:
            out = torch.empty((max(self.n_cand, 1), 4), device="cuda")
        self._check(self.lib.nbv_score(self._h, _dptr(out), 1))
        return out[: self.n_cand]

    def score_host(self):
        """Same as score() into a host array (synchronises)."""
        out = np.zeros((max(self.n_cand, 1), 4), np.float32)
        self._check(self.lib.nbv_score(self._h, ctypes.c_void_p(out.ctypes.data), 0))
        return out[: self.n_cand]

    def argmax(self):
        b = ctypes.c_int(-1)
        s = ctypes.c_float(0.0)
        self._check(self.lib.nbv_argmax(self._h, ctypes.byref(b), ctypes.byref(s)))
        return int(b.value), float(s.value)

    def set_entry_limit(self, max_entries: int):
        """Cap the (view, tile, Gaussian) entries of one binning pass (0: the
        32-bit default); see nbv_set_entry_limit."""
        self._check(self.lib.nbv_set_entry_limit(self._h, int(max_entries)))

    def train_gains(self):
        out = np.zeros((max(self.n_train, 1), 3), np.float32)
        self._check(self.lib.nbv_train_gains(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out[: self.n_train]

    def gaussian_gains(self, cand: int):
        d = self.torch.empty((self.n, 3), device="cuda")
        self._check(self.lib.nbv_gaussian_gains(self._h, int(cand), _dptr(d)))
        return d

    def debug_project(self, view_set: int, view: int):
        torch = self.torch
        n = self.n
        out = dict(rect=torch.empty((n, 4), dtype=torch.int32, device="cuda"),
                   radius=torch.empty(n, device="cuda"),
                   zbits=torch.empty(n, dtype=torch.int32, device="cuda"),
                   mean2d=torch.empty((n, 2), device="cuda"),
                   conic=torch.empty((n, 3), device="cuda"))
        self._check(self.lib.nbv_debug_project(self._h, int(view_set), int(view), _dptr(out["rect"]),
                                               _dptr(out["radius"]), _dptr(out["zbits"]),
                                               _dptr(out["mean2d"]), _dptr(out["conic"])))
        return out

    def debug_tile_lists(self, view_set: int, view: int):
        """(offsets [ntiles+1], Gaussian ids) of one view's tile lists.
        view_set 0 / 1: candidate / training view binned on its own; 2: the
        candidate as the last multi-view score binned it."""
        torch = self.torch
        cnt = ctypes.c_int64(0)
        self._check(self.lib.nbv_debug_tile_lists(self._h, int(view_set), int(view), None, None, 0,
                                                  ctypes.byref(cnt)))
        total = int(cnt.value)
        dims = self._train if view_set == 1 else self._cand
        W, H = int(dims[0][view]), int(dims[1][view])
        tw, th, _ = self.tiling()
        nt = ((W + tw - 1) // tw) * ((H + th - 1) // th)
        off = torch.empty(nt + 1, dtype=torch.int64, device="cuda")
        ids = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
        self._check(self.lib.nbv_debug_tile_lists(self._h, int(view_set), int(view), _dptr(off),
                                                  _dptr(ids), total, ctypes.byref(cnt)))
        return off, ids[:total]

    PHASES = ("prep", "project", "sort", "composite", "factors", "gains", "score", "train_composite", "forward")

    def set_profiling(self, on: bool):
        self._check(self.lib.nbv_set_profiling(self._h, 1 if on else 0))

    def phase_times(self):
        """{phase: (device ms, kernel launches)} since profiling was switched on."""
        ms = np.zeros(len(self.PHASES), np.float64)
        ln = np.zeros(len(self.PHASES), np.int64)
        self._check(self.lib.nbv_phase_times(self._h, ctypes.c_void_p(ms.ctypes.data),
                                             ctypes.c_void_p(ln.ctypes.data)))
        return {p: (float(ms[i]), int(ln[i])) for i, p in enumerate(self.PHASES)}

    def work_stats(self, training: bool = False):
        """Compositing work since profiling was switched on: the candidates'
        launches, or the training views' launches of prepare."""
        out = np.zeros(6, np.int64)
        self._check(self.lib.nbv_work_stats(self._h, 1 if training else 0, ctypes.c_void_p(out.ctypes.data)))
        return dict(pairs_evaluated=int(out[0]), pairs_blended=int(out[1]), block_flushes=int(out[2]),
                    pairs_information=int(out[3]), composite_launches=int(out[4]), entries=int(out[5]))

    def autotune(self):
        """Pick tile shape and stage depth on the batched path; returns
        (tile_w, tile_h, stage). Leaves the context prepared."""
        w, h, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.nbv_autotune(self._h, ctypes.byref(w), ctypes.byref(h), ctypes.byref(g)))
        return int(w.value), int(h.value), int(g.value)

    def tiling(self):
        w, h, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.nbv_get_tiling(self._h, ctypes.byref(w), ctypes.byref(h), ctypes.byref(g)))
        return int(w.value), int(h.value), int(g.value)

    def launch_count(self) -> int:
        return int(self.lib.nbv_launch_count(self._h))

    # ------------------------------------------------- learned pre-scoring
    DESC_DIM = 448

    def descriptors(self):
        """[n_cand, 448] per-candidate descriptors (after prepare)."""
        out = self.torch.empty((max(self.n_cand, 1), self.DESC_DIM), device="cuda")
        self._check(self.lib.nbv_descriptors(self._h, _dptr(out)))
        self.torch.cuda.synchronize()
        return out[:self.n_cand]

    def score_pruned(self, mlp, keep: int):
        """MLP pre-scores every candidate, the `keep` best are scored
        exactly; returns dict(pred, kept, exact, best, best_score)."""
        n = self.n_cand
        keep = max(1, min(int(keep), n))
        pred = self.torch.empty(max(n, 1), device="cuda")
        kept = np.zeros(keep, np.int32)
        exact = np.zeros((keep, 4), np.float32)
        best, bs = ctypes.c_int(), ctypes.c_float()
        self._check(self.lib.nbv_score_pruned(self._h, mlp._h, keep, _dptr(pred),
                                              ctypes.c_void_p(kept.ctypes.data),
                                              ctypes.c_void_p(exact.ctypes.data), ctypes.byref(best),
                                              ctypes.byref(bs)))
        return dict(pred=pred[:n], kept=kept, exact=exact, best=int(best.value), best_score=float(bs.value))


class MLP:
    """The learned candidate scorer (nbv_mlp): d_in -> width -> width -> 1,
    BF16 tensor-core layers, trained with the library's own backward and Adam."""

    def __init__(self, d_in: int = 448, width: int = 256, seed: int = 0, stream=None):
        import torch
        self.torch = torch
        self.lib = load_library()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.nbv_mlp_create(int(d_in), int(width), ctypes.c_uint64(int(seed)),
                                     ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if rc != NBV_OK:
            raise NBVError(rc, "nbv_mlp_create failed")
        self._h = h
        self.d_in, self.width = int(d_in), int(width)
        self.P = int(self.lib.nbv_mlp_num_params(h))

    def close(self):
        if getattr(self, "_h", None):
            self.lib.nbv_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != NBV_OK:
            raise NBVError(rc, what)

    def get_params(self):
        out = self.torch.empty(self.P, device="cuda")
        self._check(self.lib.nbv_mlp_get_params(self._h, _dptr(out)), "get_params")
        self.torch.cuda.synchronize()
        return out

    def set_params(self, p):
        p = p.detach().float().contiguous().cuda()
        self._check(self.lib.nbv_mlp_set_params(self._h, _dptr(p)), "set_params")
        self.torch.cuda.synchronize()

    def forward(self, x):
        x = x.detach().float().contiguous()
        y = self.torch.empty(max(x.shape[0], 1), device="cuda")
        self._check(self.lib.nbv_mlp_forward(self._h, _dptr(x), int(x.shape[0]), _dptr(y)), "forward")
        return y[:x.shape[0]]

    def gradients(self, x, t):
        x = x.detach().float().contiguous()
        t = t.detach().float().contiguous()
        g = self.torch.empty(self.P, device="cuda")
        loss = ctypes.c_double()
        self._check(self.lib.nbv_mlp_gradients(self._h, _dptr(x), _dptr(t), int(x.shape[0]), _dptr(g),
                                               ctypes.byref(loss)), "gradients")
        return g, float(loss.value)

    def train_step(self, x, t, lr: float, want_loss: bool = True):
        loss = ctypes.c_double()
        rc = self.lib.nbv_mlp_train_step(self._h, _dptr(x), _dptr(t), int(x.shape[0]), ctypes.c_float(lr),
                                         ctypes.byref(loss) if want_loss else None)
        self._check(rc, "train_step")
        return float(loss.value) if want_loss else None


def set_gemm_wait_polls(polls: int):
    """Polls of the first tensor-core wait of every GEMM launch before it
    gives up (0: at once; negative: the default); for time-out tests."""
    rc = load_library().nbv_set_gemm_wait_polls(int(polls))
    if rc != NBV_OK:
        raise NBVError(rc, "nbv_set_gemm_wait_polls")


def gemm_bf16(A, a_strides, B, b_strides, M, N, K):
    """D [M, N] float32 = sum_k A(m, k) B(n, k) on the tensor cores; A and B
    are bfloat16 CUDA tensors addressed with the given (row, k) strides."""
    import torch
    lib = load_library()
    D = torch.empty((M, N), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.nbv_gemm_bf16(_dptr(A), a_strides[0], a_strides[1], _dptr(B), b_strides[0], b_strides[1], _dptr(D),
                           N, M, N, K, _dptr(err), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != NBV_OK:
        raise NBVError(rc, "nbv_gemm_bf16")
    torch.cuda.synchronize()
    if int(err.item()) != 0:
        raise NBVError(-5, "tensor-core wait gave up")
    return D
