"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (element by element on the same seeded inputs):
  - projection key path, tile rectangles and depth bits: bit-exact;
  - tile lists: valid against the oracle's plain lists (every GPU list an
    ordered sub-list of the tile's rectangle list, holding every splat that
    passes the skip test at one of the tile's pixels): several lists are
    correct, so what is unique (the order and the needed entries) is compared
    and the rest is checked for validity;
  - colour, depth, opacity and object channels: <= 1e-4 max abs, on pixels
    whose transmittance-stop decision is not within 1e-4 (relative) of the
    threshold (those are counted and must stay rare);
  - IG per output and view: <= 1e-4 relative; the NBV argmax identical
    unless the top two totals are within 1e-4 (relative).
"""
import math

import numpy as np
import pytest

import nbv_synth as S
from oracle import oracle as O
from tests.helpers import axis_camera, make_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

IG_RTOL = 1e-4
IMG_ATOL = 1e-4


@pytest.fixture(scope="module")
def P():
    import paper_2602_08266_gb300 as P
    P.build()
    P.load_library()
    assert torch.cuda.is_available()
    return P


def _scorer(P, wl, target=-1):
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    return sc


def _ragged(wl, W=70, H=50, f=60.0):
    """A ragged-tile copy of the candidates (W, H not multiples of 16)."""
    c = wl.cand
    return S.Cameras(c.R.copy(), c.t.copy(), np.full(c.n, f, np.float32), np.full(c.n, f, np.float32),
                     np.full(c.n, W / 2, np.float32), np.full(c.n, H / 2, np.float32),
                     np.full(c.n, W, np.int32), np.full(c.n, H, np.int32))


def _check_lists_valid(goff, gids, o, cams, v):
    """GPU tile lists of view v against the oracle: each list must be an
    ordered sub-list of the tile's plain rectangle list (same (depth bits,
    index) order) and contain every splat that passes the skip test at one of
    the tile's in-image pixels. Returns (gpu entries, rectangle entries)."""
    goff = np.asarray(goff, np.int64)
    gids = np.asarray(gids, np.int64)
    off, ids = o.tile_lists(cams, v)
    noff, nids = o.tile_needed(cams, v)
    nt = len(off) - 1
    assert len(goff) == nt + 1 and goff[0] == 0 and goff[-1] == len(gids)
    N = int(o.n)
    okey = np.repeat(np.arange(nt, dtype=np.int64), np.diff(off)) * N + ids
    gkey = np.repeat(np.arange(nt, dtype=np.int64), np.diff(goff)) * N + gids
    nkey = np.repeat(np.arange(nt, dtype=np.int64), np.diff(noff)) * N + nids
    order = np.argsort(okey, kind="stable")
    sk = okey[order]
    at = np.searchsorted(sk, gkey)
    found = (at < len(sk)) & (sk[np.minimum(at, len(sk) - 1)] == gkey)
    assert found.all(), f"view {v}: {int((~found).sum())} GPU entries outside their tile's rectangle list"
    pos = order[at]
    assert (np.diff(pos) > 0).all(), f"view {v}: a GPU list is not in (depth bits, index) order"
    keep = np.isin(nkey, gkey)
    assert keep.all(), f"view {v}: {int((~keep).sum())} needed splats missing from the GPU lists"
    return len(gids), len(ids)


# --------------------------------------------------------------- key path
@pytest.mark.parametrize("ragged", [False, True])
def test_projection_keys_and_tile_lists_bit_exact(P, ragged):
    wl = S.make_workload("tiny")
    if ragged:
        wl.cand = _ragged(wl)
    sc = _scorer(P, wl)
    o = O.OracleScene(wl.scene)
    for v in range(wl.cand.n):
        g = sc.debug_project(0, v)
        r = o.project32(wl.cand, v)
        rect = g["rect"].cpu().numpy()
        np.testing.assert_array_equal(rect, r["rect"])
        ok = r["rect"][:, 0] >= 0
        np.testing.assert_array_equal(g["zbits"].cpu().numpy().view(np.uint32)[ok], r["zbits"][ok])
        np.testing.assert_array_equal(g["radius"].cpu().numpy()[ok], r["radius"][ok])
        np.testing.assert_array_equal(g["mean2d"].cpu().numpy()[ok], r["mean2d"][ok])
        np.testing.assert_array_equal(g["conic"].cpu().numpy()[ok], r["conic"][ok])
        off, ids = sc.debug_tile_lists(0, v)
        _check_lists_valid(off.cpu().numpy(), ids.cpu().numpy(), o, wl.cand, v)


# ---------------------------------------------------------------- renders
def _compare_render(sc, o, cams, v, K):
    g = {k: t.cpu().numpy().astype(np.float64) for k, t in sc.render(v).items()}
    r = o.render(cams, v)
    ok = r["margin"] >= 1e-4
    frac_flag = 1.0 - ok.mean()
    assert frac_flag < 0.01, frac_flag
    for k in ("rgb", "depth", "alpha", "obj"):
        d = np.abs(g[k] - r[k])
        if d.ndim == 3:
            d = d.max(-1)
        assert d[ok].max() <= IMG_ATOL, (k, v, d[ok].max())
    return frac_flag


@pytest.mark.parametrize("ragged", [False, True])
def test_render_parity_tiny(P, ragged):
    wl = S.make_workload("tiny")
    if ragged:
        wl.cand = _ragged(wl)
    sc = _scorer(P, wl)
    o = O.OracleScene(wl.scene)
    for v in range(wl.cand.n):
        _compare_render(sc, o, wl.cand, v, wl.scene.K)


def test_render_parity_scene_scale_one_view(P):
    """Full scene-scale workload (120k Gaussians, SH degree 3, K=16,
    640x480): keys bit-exact, tile lists valid, render within tolerance."""
    wl = S.make_workload("scene", n_views=2)
    sc = _scorer(P, wl)
    o = O.OracleScene(wl.scene)
    v = 1
    g = sc.debug_project(0, v)
    r = o.project32(wl.cand, v)
    np.testing.assert_array_equal(g["rect"].cpu().numpy(), r["rect"])
    off, ids = sc.debug_tile_lists(0, v)
    n_gpu, n_rect = _check_lists_valid(off.cpu().numpy(), ids.cpu().numpy(), o, wl.cand, v)
    assert n_gpu < n_rect                       # the tile culling drops entries
    _compare_render(sc, o, wl.cand, v, wl.scene.K)


# ------------------------------------------------------------------- IG
def _check_scores(gpu4, ref, train_gpu=None, rtol=IG_RTOL):
    igc = ref["ig_cand"]
    np.testing.assert_allclose(gpu4[:, :3], igc, rtol=rtol, atol=0)
    if train_gpu is not None:
        np.testing.assert_allclose(train_gpu, ref["ig_train"], rtol=rtol, atol=0)
    tot = ref["score"]
    np.testing.assert_allclose(gpu4[:, 3], tot, rtol=rtol)
    order = np.argsort(-tot)
    best_g = int(np.argmax(gpu4[:, 3]))
    if len(tot) > 1 and (tot[order[0]] - tot[order[1]]) > 2 * rtol * abs(tot[order[0]]):
        assert best_g == ref["best"]


@pytest.mark.parametrize("target", [-1, 2])
def test_ig_parity_tiny(P, target):
    wl = S.make_workload("tiny")
    sc = _scorer(P, wl)
    sc.prepare(target)
    g4 = sc.score_host().astype(np.float64)
    best, bs = sc.argmax()
    ref = O.OracleScene(wl.scene, target=target).score(wl.train, wl.cand)
    _check_scores(g4, ref, sc.train_gains().astype(np.float64))
    assert best == int(np.argmax(g4[:, 3]))


def test_per_gaussian_gains_tiny(P):
    wl = S.make_workload("tiny")
    sc = _scorer(P, wl)
    sc.prepare(-1)
    v = 3
    d = sc.gaussian_gains(v).cpu().numpy().astype(np.float64)
    ref = O.OracleScene(wl.scene).score(wl.train, wl.cand, delta_view=v)["delta"]
    assert (d >= -1e-6).all()
    from tests.test_gpu_golden import check_gaussian_gains
    check_gaussian_gains(d, ref, wl.scene.K)
    np.testing.assert_allclose(d.sum(0), ref.sum(0), rtol=IG_RTOL)


def test_ig_parity_ragged_and_sh_degree_3(P):
    """SH degree 3, K = 6, ragged 70x50 views: exercises the colour
    direction Jacobian and partial tiles."""
    wl = S.make_workload("tiny")
    rng = np.random.default_rng(5)
    sc0 = wl.scene
    sh = np.zeros((sc0.n, 16, 3), np.float32)
    sh[:, 0, :] = sc0.sh[:, 0, :]
    sh[:, 1:, :] = rng.normal(0, 0.1, (sc0.n, 15, 3))
    K = 6
    obj = np.zeros((sc0.n, K + 1), np.float32)
    obj[:, : sc0.K + 1] = sc0.obj_logits
    wl.scene = S.Scene(sc0.means, sc0.log_scales, sc0.quats, sc0.opacity, sh, obj, 3, K)
    wl.cand = _ragged(wl)
    wl.train = S.training_cameras(70, 50, 60.0)
    sc = _scorer(P, wl)
    sc.prepare(-1)
    ref = O.OracleScene(wl.scene).score(wl.train, wl.cand)
    _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))


def test_ig_parity_scene_scale_reduced(P):
    """The scene-scale structure (blobs + table, SH 3, K=16) with a
    twentieth of the Gaussians at 320x240 (f = 262.5), 2 training views and
    2 candidates: sized so that the oracle finishes in well under a minute."""
    wl = S.make_workload("scene", n_views=2, scale=0.05)
    wl.cand = _ragged(wl, 320, 240, 262.5)
    wl.train = S.training_cameras(320, 240, 262.5).subset([0, 2])
    sc = _scorer(P, wl)
    sc.prepare(-1)
    ref = O.OracleScene(wl.scene).score(wl.train, wl.cand)
    _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))


# ------------------------------------------------------------- edge cases
def test_empty_view_and_single_pixel(P):
    wl = S.make_workload("tiny")
    away = S.Cameras(np.eye(3, dtype=np.float32)[None], np.array([[0, 0, -5.0]], np.float32),
                     np.array([60.0], np.float32), np.array([60.0], np.float32),
                     np.array([32.0], np.float32), np.array([24.0], np.float32),
                     np.array([64], np.int32), np.array([48], np.int32))
    one = axis_camera(1, 1, 60.0, 0.6)
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(S.Cameras.concat([away, one]))
    sc.prepare(-1)
    g4 = sc.score_host()
    assert np.all(g4[0, :3] == 0.0)                       # nothing visible: no gain
    r = sc.render(0)
    assert float(r["alpha"].abs().max()) == 0.0
    assert float((r["obj"][..., 0] - 1).abs().max()) == 0.0   # all background
    o = O.OracleScene(wl.scene)
    ref = o.score(wl.train, S.Cameras.concat([away, one]))
    np.testing.assert_allclose(g4[:, :3], ref["ig_cand"], rtol=IG_RTOL, atol=1e-9)


def test_target_without_gaussians_is_empty(P):
    wl = S.make_workload("tiny")
    wl.scene.obj_logits[:, 3] = -5.0
    sc = _scorer(P, wl)
    sc.prepare(3)
    with pytest.raises(P.NBVError) as e:
        sc.score_host()
    assert e.value.code == -6
    with pytest.raises(P.NBVError):
        sc.argmax()


def test_invalid_inputs_are_rejected(P):
    wl = S.make_workload("tiny")
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree)
    q = wl.scene.quats.copy(); q[5] = 0
    with pytest.raises(P.NBVError) as e:
        sc.load_gaussians(wl.scene.means, wl.scene.log_scales, q, wl.scene.opacity, wl.scene.sh,
                          wl.scene.obj_logits)
    assert e.value.code == -1
    m = wl.scene.means.copy(); m[3, 1] = np.nan
    with pytest.raises(P.NBVError):
        sc.load_gaussians(m, wl.scene.log_scales, wl.scene.quats, wl.scene.opacity, wl.scene.sh,
                          wl.scene.obj_logits)
    sc.load_scene(wl.scene)
    with pytest.raises(P.NBVError) as e:
        sc.prepare(-1)                                     # no training views yet
    assert e.value.code == -4
    sc.set_train_views(wl.train)
    with pytest.raises(P.NBVError) as e:
        sc.prepare(wl.scene.K + 1)
    assert e.value.code == -1


def test_device_inputs_match_host_inputs(P):
    wl = S.make_workload("tiny")
    a = _scorer(P, wl)
    a.prepare(-1)
    ga = a.score_host()
    b = P.NBVScorer(wl.scene.K, wl.scene.sh_degree)
    sc = wl.scene
    b.load_gaussians(*[torch.from_numpy(x).cuda() for x in
                       (sc.means, sc.log_scales, sc.quats, sc.opacity, sc.sh, sc.obj_logits)])
    b.set_train_views(wl.train)
    b.set_candidates(wl.cand)
    b.prepare(-1)
    gb = b.score_host()
    np.testing.assert_allclose(ga, gb, rtol=1e-6)


# ------------------------------------------------------------ batched path
def _mixed(wl):
    """Alternating 70x50 (f 60) and 64x48 (f 60) candidates: several tile
    grids in one multi-view launch."""
    c = wl.cand
    W = np.where(np.arange(c.n) % 2 == 0, 70, 64).astype(np.int32)
    H = np.where(np.arange(c.n) % 2 == 0, 50, 48).astype(np.int32)
    return S.Cameras(c.R.copy(), c.t.copy(), c.fx.copy(), c.fy.copy(), (W / 2).astype(np.float32),
                     (H / 2).astype(np.float32), W, H)


@pytest.mark.parametrize("mixed,target", [(False, -1), (True, -1), (True, 1)])
def test_batched_ig_parity_tiny(P, mixed, target):
    wl = S.make_workload("tiny")
    if mixed:
        wl.cand = _mixed(wl)
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    sc.prepare(target)
    ref = O.OracleScene(wl.scene, target=target).score(wl.train, wl.cand)
    for _ in range(2):                       # capture, then graph replay
        g4 = sc.score_host().astype(np.float64)
        _check_scores(g4, ref, sc.train_gains().astype(np.float64))
        best, _ = sc.argmax()
        assert best == int(np.argmax(g4[:, 3]))


def test_batched_matches_per_view_scene_scale_and_recaptures(P):
    """The full scene-scale workload scored by the per-view path and by the
    batched graph path agree to 1e-4; changing the candidate set recaptures."""
    wl = S.make_workload("scene", n_views=16)
    a = _scorer(P, wl)
    a.prepare(-1)
    ga = a.score_host().astype(np.float64)
    a.close()
    b = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
    b.load_scene(wl.scene)
    b.set_train_views(wl.train)
    b.set_candidates(wl.cand)
    b.prepare(-1)
    for _ in range(2):
        gb = b.score_host().astype(np.float64)
        np.testing.assert_allclose(gb, ga, rtol=1e-4)
    b.set_candidates(wl.cand.subset(np.arange(8)))
    gc = b.score_host().astype(np.float64)
    np.testing.assert_allclose(gc, ga[:8], rtol=1e-4)


# ------------------------------------------------- tile shape / stage depth
@pytest.mark.parametrize("batched", [0, 1])
def test_tile_32x8_parity_tiny(P, batched):
    """32 x 8 screen tiles: keys, tile lists and renders against the oracle
    run with the same tile shape (ragged grids), and IG on both paths."""
    wl = S.make_workload("tiny")
    wl.cand = _mixed(wl)
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, tile_w=32, tile_h=8, batched=batched)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    assert sc.tiling()[:2] == (32, 8)
    o = O.OracleScene(wl.scene, hyper=O.Hyper(tile_w=32, tile_h=8))
    for v in range(wl.cand.n):
        g = sc.debug_project(0, v)
        r = o.project32(wl.cand, v)
        np.testing.assert_array_equal(g["rect"].cpu().numpy(), r["rect"])
        off, ids = sc.debug_tile_lists(0, v)
        _check_lists_valid(off.cpu().numpy(), ids.cpu().numpy(), o, wl.cand, v)
        _compare_render(sc, o, wl.cand, v, wl.scene.K)
    sc.prepare(-1)
    ref = o.score(wl.train, wl.cand)
    for _ in range(2):
        _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))


def test_stage_depth_changes_nothing_but_speed(P):
    """Staging 16 instead of 32 Gaussians per shared-memory round leaves the
    gains equal up to float summation order."""
    wl = S.make_workload("scene", n_views=6, scale=0.05)
    out = []
    for stage in (32, 16):
        sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1, stage=stage)
        sc.load_scene(wl.scene)
        sc.set_train_views(wl.train)
        sc.set_candidates(wl.cand)
        assert sc.tiling()[2] == stage
        sc.prepare(-1)
        out.append(sc.score_host().astype(np.float64))
        sc.close()
    np.testing.assert_allclose(out[1], out[0], rtol=1e-4)


def test_autotune_picks_a_valid_tiling_and_scores_match_oracle(P):
    wl = S.make_workload("tiny")
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    sc.prepare(-1)
    tw, th, st = sc.autotune()
    assert (tw, th) in ((16, 16), (32, 8)) and st in (16, 32)
    assert sc.tiling() == (tw, th, st)
    ref = O.OracleScene(wl.scene, hyper=O.Hyper(tile_w=tw, tile_h=th)).score(wl.train, wl.cand)
    _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))
    sc2 = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)   # cached choice
    sc2.load_scene(wl.scene)
    sc2.set_train_views(wl.train)
    sc2.set_candidates(wl.cand)
    assert sc2.autotune() == (tw, th, st)


@pytest.mark.parametrize("name,n_views,views", [("tiny", 8, None), ("scene", 6, (0, 5)), ("scene", 64, (0, 37, 63))])
def test_batched_tile_lists_valid(P, name, n_views, views):
    """The multi-view binning (depth order of all (view, Gaussian) slots,
    duplication in that order, stable sort on the 32-bit tile id) gives
    every candidate valid lists: ordered sub-lists of the oracle's
    (depth bits, index) rectangle lists holding every needed splat. With 64
    views at 640x480 the tile ids take 17 bits (a third radix pass)."""
    wl = S.make_workload(name, n_views=n_views)
    if name == "tiny":
        wl.cand = _mixed(wl)
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    sc.prepare(-1)
    sc.score_host()
    o = O.OracleScene(wl.scene)
    for v in (views if views is not None else range(wl.cand.n)):
        off, ids = sc.debug_tile_lists(2, v)
        _check_lists_valid(off.cpu().numpy(), ids.cpu().numpy(), o, wl.cand, v)
        # the per-view binning of the same candidate gives the same lists
        off1, ids1 = sc.debug_tile_lists(0, v)
        np.testing.assert_array_equal(off1.cpu().numpy(), off.cpu().numpy())
        np.testing.assert_array_equal(ids1.cpu().numpy(), ids.cpu().numpy())
    sc.close()


def test_batched_chunks_match_single_pass(P):
    """A candidate set scored in multi-view chunks of 3 (eagerly, one chunk
    after the other) equals the single-pass graph path and the oracle; the
    last chunk's tile lists stay inspectable."""
    wl = S.make_workload("tiny")
    wl.cand = _mixed(wl)
    out = []
    for mbv in (0, 3):
        sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1, max_batch_views=mbv)
        sc.load_scene(wl.scene)
        sc.set_train_views(wl.train)
        sc.set_candidates(wl.cand)
        sc.prepare(-1)
        out.append(sc.score_host().astype(np.float64))
        out.append(sc.score_host().astype(np.float64))
        if mbv == 3:
            off, ids = sc.debug_tile_lists(2, wl.cand.n - 1)
            _check_lists_valid(off.cpu().numpy(), ids.cpu().numpy(), O.OracleScene(wl.scene), wl.cand,
                               wl.cand.n - 1)
        sc.close()
    for o in out[1:]:
        np.testing.assert_allclose(o, out[0], rtol=1e-5)
    ref = O.OracleScene(wl.scene).score(wl.train, wl.cand)
    _check_scores(out[2], ref)


@pytest.mark.parametrize("crit,batched,target", [(1, 0, -1), (1, 1, 2), (2, 0, -1), (2, 1, -1)])
def test_criterion_variants_parity(P, crit, batched, target):
    """tr(H_T^-1 c A) (crit 1) and T-optimality tr(c A) (crit 2) on the
    per-view and multi-view paths against the oracle at 1e-4 relative. Both
    are linear in the 2D blocks, so the automatic contraction mode gives
    them error-compensated products (three TF32 products per term)."""
    wl = S.make_workload("tiny")
    wl.cand = _mixed(wl)
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=batched, criterion=crit)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    sc.prepare(target)
    ref = O.OracleScene(wl.scene, hyper=O.Hyper(crit=crit), target=target).score(wl.train, wl.cand)
    _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))
    sc.close()


@pytest.mark.parametrize("batched", [0, 1])
def test_contraction_modes_log_det_parity(P, batched):
    """The log-det gains (criterion 0) with single TF32 products (mode 1, the
    automatic choice for this criterion) and with error-compensated products
    (mode 2): both within 1e-4 relative of the oracle, and of each other."""
    wl = S.make_workload("tiny")
    out = []
    for mode in (2, 1):
        sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=batched, tf32_contraction=mode)
        sc.load_scene(wl.scene)
        sc.set_train_views(wl.train)
        sc.set_candidates(wl.cand)
        sc.prepare(-1)
        out.append(sc.score_host().astype(np.float64))
        sc.close()
    ref = O.OracleScene(wl.scene).score(wl.train, wl.cand)
    for o in out:
        _check_scores(o, ref)
    np.testing.assert_allclose(out[1], out[0], rtol=1e-4)


@pytest.mark.slow
def test_batched_target_tile_lists_valid(P):
    """With a target object (Eq. 12) the multi-view pass bins only the tiles
    where a splat of the target can pass its alpha cut-off (marked by the
    active slots' projection), drops slots whose rectangle cannot reach the
    view's box of such tiles before their key path, and duplicates the
    survivors' tiles in packed warp rounds. Its lists must still be ordered
    sub-lists of the oracle's rectangle lists, and every tile where the
    oracle finds a target splat passing the skip test at an in-image pixel
    must hold every splat (target or not) needed there."""
    wl = S.make_workload("batch", n_views=6, scale=0.05)
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    sc.prepare(wl.target)
    sc.score_host()
    o = O.OracleScene(wl.scene, target=wl.target)
    act = o.confidence() > 0
    assert 0 < act.sum() < wl.scene.n
    for v in range(wl.cand.n):
        off, ids = sc.debug_tile_lists(2, v)
        goff, gids = off.cpu().numpy().astype(np.int64), ids.cpu().numpy().astype(np.int64)
        roff, rids = o.tile_lists(wl.cand, v)
        noff, nids = o.tile_needed(wl.cand, v)
        nt = len(roff) - 1
        assert len(goff) == nt + 1 and goff[-1] == len(gids)
        N = wl.scene.n
        rkey = np.repeat(np.arange(nt), np.diff(roff)) * N + rids
        gkey = np.repeat(np.arange(nt), np.diff(goff)) * N + gids
        ntile = np.repeat(np.arange(nt), np.diff(noff))
        order = np.argsort(rkey, kind="stable")
        sk = rkey[order]
        at = np.searchsorted(sk, gkey)
        assert ((at < len(sk)) & (sk[np.minimum(at, len(sk) - 1)] == gkey)).all(), v
        assert (np.diff(order[at]) > 0).all(), v
        target_tiles = np.unique(ntile[act[nids]])
        need = np.isin(ntile, target_tiles)
        assert need.any(), v
        assert np.isin(ntile[need] * N + nids[need], gkey).all(), v
    sc.close()


def test_batch_workload_full_size():
    """The batching workload at full size (300k Gaussians, K = 32, 256
    candidates alternating 320x240 / 640x480, IG restricted to object 1),
    scored on the multi-view path: a sample of candidates equals the
    per-view path; two candidates' tile lists are valid against the
    oracle's and one candidate's render matches the oracle's."""
    import paper_2602_08266_gb300 as P
    P.build()
    wl = S.make_workload("batch")
    assert wl.scene.n == 300_000 and wl.cand.n == 256 and wl.target == 1
    b = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
    b.load_scene(wl.scene)
    b.set_train_views(wl.train)
    b.set_candidates(wl.cand)
    b.prepare(wl.target)
    gb = b.score_host().astype(np.float64)
    assert np.all(np.isfinite(gb)) and (gb[:, :3] >= 0).all()
    o = O.OracleScene(wl.scene, target=wl.target)
    sample = np.array([0, 1, 97, 254, 255])
    a = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=0)
    a.load_scene(wl.scene)
    a.set_train_views(wl.train)
    a.set_candidates(wl.cand.subset(sample))
    a.prepare(wl.target)
    ga = a.score_host().astype(np.float64)
    np.testing.assert_allclose(gb[sample], ga, rtol=1e-4)
    for v in (1, 254):
        off, ids = a.debug_tile_lists(0, int(np.nonzero(sample == v)[0][0]))
        _check_lists_valid(off.cpu().numpy(), ids.cpu().numpy(), o, wl.cand, v)
    _compare_render(a, o, wl.cand.subset(sample), 3, wl.scene.K)
    a.close()
    b.close()


# --------------------------------------------------------- entry-count guard
def test_entry_limit_splits_batched_passes_and_rejects_single_views(P):
    """The entries of a binning pass are counted in 64 bits before anything
    is duplicated: under a small forced limit the batched path splits its
    candidates into smaller passes (same scores), and a single view above
    the limit is refused with NBV_ERR_ARG on both paths (nothing written)."""
    wl = S.make_workload("tiny")
    wl.cand = _mixed(wl)
    counts = []
    a = _scorer(P, wl)
    for v in range(wl.cand.n):
        off, _ = a.debug_tile_lists(0, v)
        counts.append(int(off[-1]))
    a.prepare(-1)
    want = a.score_host().astype(np.float64)
    b = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
    b.load_scene(wl.scene)
    b.set_train_views(wl.train)
    b.set_candidates(wl.cand)
    b.prepare(-1)
    b.set_entry_limit(int(2.5 * max(counts)))         # at most two views per pass
    assert sum(counts) > 2.5 * max(counts)
    for _ in range(2):
        np.testing.assert_allclose(b.score_host().astype(np.float64), want, rtol=1e-5)
    b.set_entry_limit(max(counts) - 1)                 # the largest view alone is too many
    with pytest.raises(P.NBVError) as e:
        b.score_host()
    assert e.value.code == -1
    a.set_entry_limit(max(counts) - 1)
    with pytest.raises(P.NBVError) as e:
        a.score_host()
    assert e.value.code == -1
    a.set_entry_limit(0)                               # default restored
    np.testing.assert_allclose(a.score_host().astype(np.float64), want, rtol=1e-6)
    with pytest.raises(P.NBVError):
        a.set_entry_limit(-5)
    a.close()
    b.close()


# ------------------------------------------------------------ single object
@pytest.mark.parametrize("batched", [0, 1])
def test_single_object_k1_parity(P, batched):
    """K = 1 (two object channels: the object and the background): renders
    within 1e-4 and IG within 1e-4 relative with the oracle's argmax, with
    and without the object as the target (Eq. 12)."""
    wl = S.make_workload("tiny")
    sc0 = wl.scene
    obj = np.stack([sc0.obj_logits[:, 0], sc0.obj_logits[:, 1:].max(1)], 1).astype(np.float32)
    wl.scene = S.Scene(sc0.means, sc0.log_scales, sc0.quats, sc0.opacity, sc0.sh, obj, sc0.sh_degree, 1)
    sc = P.NBVScorer(1, wl.scene.sh_degree, batched=batched)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    o = O.OracleScene(wl.scene)
    for v in (0, 5):
        _compare_render(sc, o, wl.cand, v, 1)
    for target in (-1, 1):
        sc.prepare(target)
        ref = O.OracleScene(wl.scene, target=target).score(wl.train, wl.cand)
        _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))
    sc.close()


# ------------------------------------------------- culling of elongated splats
@pytest.mark.parametrize("aniso", [0.25, 2.5])
def test_tile_culling_elongated_splats_valid(P, aniso):
    """The GPU's ellipse-tile culling on splats with axis ratios beyond 1000
    (log-scale spread 2.5), where cancellation in the exponent is largest:
    every list still holds every splat that passes the skip test at one of
    the tile's pixels. Renders are compared on the moderate scene only: at
    axis ratios beyond 1000 the single-precision conic (its determinant
    a c - b^2 cancels) moves the rendered values by more than 1e-4 from the
    double-precision definition, a limit of single-precision projection that
    the tile lists do not depend on."""
    rng = np.random.default_rng(7)
    n = 400
    means = np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(-0.1, 0.3, n)], 1)
    log_scales = rng.normal(np.log(0.01), aniso, (n, 3))
    q = rng.standard_normal((n, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = rng.normal(0.0, 1.5, n)
    sh = np.zeros((n, 1, 3)); sh[:, 0, :] = 0.8
    obj = rng.normal(0, 1.0, (n, 2))
    scene = make_scene(means, log_scales, q, opacity, sh, obj, 1, 0)
    cam = axis_camera(200, 152, 180.0, 1.0)
    for tw, th in ((16, 16), (32, 8)):
        sc = P.NBVScorer(1, 0, tile_w=tw, tile_h=th)
        sc.load_scene(scene)
        sc.set_candidates(cam)
        o = O.OracleScene(scene, hyper=O.Hyper(tile_w=tw, tile_h=th))
        off, ids = sc.debug_tile_lists(0, 0)
        n_gpu, n_rect = _check_lists_valid(off.cpu().numpy(), ids.cpu().numpy(), o, cam, 0)
        assert n_gpu < n_rect
        if aniso < 1.0:
            _compare_render(sc, o, cam, 0, 1)
        sc.close()


def test_batch_workload_reduced_target_parity(P):
    """The batching workload's structure (32 blobs + table, K = 32, SH 3,
    candidates alternating 320x240 and 640x480, object-centric on object 1,
    Eq. 12) with a fiftieth of the Gaussians, 2 candidates and the training
    views at 320x240 (so that the oracle finishes in about a minute): the
    multi-view graph path (tiles an active splat reaches are the only ones
    binned) and the per-view path against the oracle at 1e-4."""
    wl = S.make_workload("batch", n_views=2, scale=0.02)
    wl.train = S.training_cameras(320, 240, 262.5)
    assert wl.target == 1 and set(wl.cand.width.tolist()) == {320, 640}
    ref = O.OracleScene(wl.scene, target=wl.target).score(wl.train, wl.cand)
    for batched in (1, 0):
        sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=batched)
        sc.load_scene(wl.scene)
        sc.set_train_views(wl.train)
        sc.set_candidates(wl.cand)
        sc.prepare(wl.target)
        for _ in range(2 if batched else 1):
            _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))
        sc.close()


@pytest.mark.parametrize("crit,batched", [(0, 1), (1, 1), (0, 0)])
def test_k32_object_gains_parity(P, crit, batched):
    """K = 32 objects (the object block of a Gaussian is 38 x 38, eliminated
    two rows per lane) on the tiny scene with its logits padded to 33
    channels: log-det and first-order trace gains against the oracle."""
    wl = S.make_workload("tiny")
    sc0 = wl.scene
    K = 32
    rng = np.random.default_rng(11)
    obj = rng.normal(-1.0, 0.5, (sc0.n, K + 1)).astype(np.float32)
    obj[:, : sc0.K + 1] = sc0.obj_logits
    wl.scene = S.Scene(sc0.means, sc0.log_scales, sc0.quats, sc0.opacity, sc0.sh, obj, sc0.sh_degree, K)
    sc = P.NBVScorer(K, wl.scene.sh_degree, batched=batched, criterion=crit)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    sc.prepare(-1)
    ref = O.OracleScene(wl.scene, hyper=O.Hyper(crit=crit)).score(wl.train, wl.cand)
    _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))
    sc.close()


@pytest.mark.parametrize("K", [48, 98])
def test_many_objects_parity(P, K):
    """K = 48 and K = 98, the largest the library takes: the object block of
    a Gaussian is u x u with u = 6 + K > 40, factorised by the generic
    elimination, the multi-view gains fall back to the view-major kernel
    where a warp's Gaussian-major layout does not fit, and at K = 98 the
    compositing kernel runs its widest variant (128 object channels) at 16
    splats a round. A quarter of the tiny scene with its logits padded to
    K + 1 channels and 3 candidates; per-view and multi-view paths against
    the oracle at the IG tolerance."""
    wl = S.make_workload("tiny", n_views=3, scale=0.25)
    sc0 = wl.scene
    rng = np.random.default_rng(K)
    obj = rng.normal(-1.0, 0.5, (sc0.n, K + 1)).astype(np.float32)
    obj[:, : sc0.K + 1] = sc0.obj_logits
    scene = S.Scene(sc0.means, sc0.log_scales, sc0.quats, sc0.opacity, sc0.sh, obj, sc0.sh_degree, K)
    ref = O.OracleScene(scene).score(wl.train, wl.cand)
    for batched in (0, 1):
        sc = P.NBVScorer(K, scene.sh_degree, batched=batched)
        sc.load_scene(scene)
        sc.set_train_views(wl.train)
        sc.set_candidates(wl.cand)
        sc.prepare(-1)
        _check_scores(sc.score_host().astype(np.float64), ref, sc.train_gains().astype(np.float64))
        sc.close()
