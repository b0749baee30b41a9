"""CPU-side checks of the product library: it builds for sm_103a, loads, and
exports every entry point include/nbvgs.h declares (no GPU call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2602_08266_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nbvgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nbv_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = P.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # the binding covers the whole ABI
    assert sorted(P.exported_symbols()) == names


def test_config_defaults_are_the_papers():
    from tests.helpers import paper_hyperparameters
    P.build()
    cfg = P.config_default(16, 3)
    assert cfg.K == 16 and cfg.sh_degree == 3
    for name, value in paper_hyperparameters().items():
        assert getattr(cfg, name) == np.float32(value), name
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and abs(cfg.t_min - 1e-4) < 1e-10
    assert cfg.tile_w == 16 and cfg.tile_h == 16 and cfg.stage == 32 and cfg.batched == 0


def test_create_rejects_bad_config_without_gpu():
    P.build()
    lib = P.load_library()
    # K = 99: the object gain's workspace does not fit a block's shared memory
    for kw in (dict(K=0), dict(K=99), dict(sh_degree=4), dict(tile_w=8), dict(tile_w=32), dict(stage=24),
               dict(lambda_damp=0.0), dict(alpha_max=1.0)):
        cfg = P.config_default(4, 0)
        for k, v in kw.items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        assert lib.nbv_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
