"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test checks the oracle against something the paper or the mathematics
fixes: closed forms, a hand-worked occlusion case, finite differences of its
own rendered outputs, brute force at tiny sizes, library eigen-solvers, and
the invariants the paper states (Sigma_k O_k = 1 from Eq. 2, a training view
scoring exactly one per output after Eq. 10, Eq. 12 zeroing non-target
Gaussians).
"""
import math

import numpy as np
import pytest

import nbv_synth as S
from oracle import oracle as O
from tests.helpers import axis_camera, make_scene, random_small_scene

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


# --------------------------------------------------------------- SH basis
def test_sh_orthonormal_on_sphere():
    """Real SH up to degree 3 are orthonormal on the unit sphere
    (Gauss-Legendre in cos(theta) x uniform in phi, exact for these degrees)."""
    nt, nphi = 16, 32
    x, wx = np.polynomial.legendre.leggauss(nt)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wx[:, None] * np.full((1, nphi), 2 * np.pi / nphi)).reshape(-1)
    Y = O.sh_basis(3, dirs)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_low_order_convention():
    """Y_00 = 1/(2 sqrt(pi)); degree 1 is (-y, z, -x) sqrt(3/(4 pi))."""
    rng = np.random.default_rng(1)
    d = rng.standard_normal((50, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = O.sh_basis(1, d)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[:, 0], Y00, rtol=1e-14)
    np.testing.assert_allclose(Y[:, 1], -c1 * d[:, 1], atol=1e-14)
    np.testing.assert_allclose(Y[:, 2], c1 * d[:, 2], atol=1e-14)
    np.testing.assert_allclose(Y[:, 3], -c1 * d[:, 0], atol=1e-14)


def test_sh_degree_l_is_harmonic_polynomial():
    """r^l Y_lm is a homogeneous harmonic polynomial of degree l: its
    Laplacian (central differences of the homogeneous extension) vanishes."""
    rng = np.random.default_rng(2)
    p = rng.standard_normal((20, 3)) * 0.7
    h = 1e-3

    def ext(q):
        r = np.linalg.norm(q, axis=1)
        Y = O.sh_basis(3, q / r[:, None])
        ls = np.array([int(math.isqrt(k)) for k in range(16)])
        return Y * r[:, None] ** ls[None, :]

    lap = -6 * ext(p)
    for a in range(3):
        e = np.zeros(3); e[a] = h
        lap = lap + ext(p + e) + ext(p - e)
    lap /= h * h
    assert np.abs(lap).max() < 1e-4


# ------------------------------------------------------ confidence, Eqs. 7 and 12
def test_oracle_defaults_are_the_printed_hyperparameters():
    from tests.helpers import paper_hyperparameters
    h = O.Hyper()
    for name, value in paper_hyperparameters().items():
        assert getattr(h, name) == value, name


def test_confidence_eq7_eq12_hand_values():
    # K = 1: logits [0, log 3] -> p = [1/4, 3/4]; rho = 0 -> sigma = 1/2
    sc = make_scene([[0, 0, 0], [0, 0, 0.01], [0, 0, 0.02]], np.full((3, 3), math.log(0.01)),
                    opacity=[0.0, 0.0, math.log(3.0)],
                    obj=[[0.0, math.log(3.0)], [1.0, 1.0], [math.log(4.0), 0.0]], K=1)
    whole = O.OracleScene(sc).confidence()
    exp0 = 0.75 ** -0.3 * 0.5 ** -0.3
    exp1 = 0.5 ** -0.3 * 0.5 ** -0.3
    exp2 = 0.8 ** -0.3 * 0.75 ** -0.3
    np.testing.assert_allclose(whole, [exp0, exp1, exp2], rtol=2e-7)
    t1 = O.OracleScene(sc, target=1).confidence()
    # Gaussian 1 has a tie: argmax goes to the lowest id (0), not the target
    np.testing.assert_allclose(t1, [exp0, 0.0, 0.0], rtol=2e-7)
    t0 = O.OracleScene(sc, target=0).confidence()
    np.testing.assert_allclose(t0, [0.0, 0.5 ** -0.3 * 0.5 ** -0.3, 0.8 ** -0.3 * 0.75 ** -0.3],
                               rtol=2e-7)


# ------------------------------------------------- single isotropic splat
def _iso(s=0.05, sigma=0.3, z0=0.5, rgb=(0.2, 0.5, 0.9), K=1):
    rho = math.log(sigma / (1 - sigma))
    sh = np.zeros((1, 1, 3)); sh[0, 0, :] = (np.array(rgb) - 0.5) / Y00
    sc = make_scene([[0, 0, 0]], [[math.log(s)] * 3], opacity=[rho], sh=sh,
                    obj=[[0.0, 1.0]], K=K)
    return sc, axis_camera(64, 64, 60.0, z0)


def test_single_isotropic_splat_integral():
    """Sum of alpha over pixels ~ integral 2 pi s2^2 (sigma - 1/255) of the
    truncated Gaussian, s2^2 = (f s/z)^2 + 0.3 (EWA on the optical axis)."""
    s, sigma, z0, f = 0.05, 0.3, 0.5, 60.0
    sc, cam = _iso(s, sigma, z0)
    r = O.OracleScene(sc).render(cam, 0)
    sig32 = float(np.float32(1.0 / (1.0 + math.exp(-math.log(sigma / (1 - sigma))))))
    s2sq = (f * float(np.float32(s)) / z0) ** 2 + float(np.float32(0.3))
    integral = 2 * math.pi * s2sq * (sig32 - 1 / 255)
    r_c = math.sqrt(s2sq) * math.sqrt(2 * math.log(255 * sig32))
    assert 3 * math.sqrt(s2sq) > r_c                         # 3-sigma rect covers the disc
    edge = 2 * math.pi * r_c / 255                           # jump at the cut-off circle
    assert abs(r["alpha"].sum() - integral) < edge
    # the nearest pixel centre to the splat centre (32,32) is 0.5 px off per axis
    a_peak = sig32 * math.exp(-0.5 * (0.25 + 0.25) / s2sq)
    np.testing.assert_allclose(r["alpha"][31, 31], a_peak, rtol=1e-6)
    # one Gaussian: D = z A, C = rgb A, O' = p A and O_0 takes the residual
    np.testing.assert_allclose(r["depth"], z0 * r["alpha"], rtol=1e-6, atol=1e-12)
    rgb = (np.array([0.2, 0.5, 0.9], np.float32) - 0.5) / np.float32(Y00)
    rgb = rgb.astype(np.float32).astype(np.float64) * Y00 + 0.5
    np.testing.assert_allclose(r["rgb"], r["alpha"][..., None] * rgb, rtol=1e-6, atol=1e-12)
    p1 = math.e / (1 + math.e)
    np.testing.assert_allclose(r["obj"][..., 1], p1 * r["alpha"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["obj"][..., 0], 1 - p1 * r["alpha"], rtol=1e-12)


def test_alpha_clamp_and_cutoff():
    """An opaque splat clamps at alpha = 0.99; nothing below 1/255 is blended."""
    sc, cam = _iso(s=0.05, sigma=0.9995)
    r = O.OracleScene(sc).render(cam, 0)
    assert r["alpha"].max() == float(np.float32(0.99))     # the clamp is the float 0.99
    a = r["alpha"][r["alpha"] > 0]
    assert a.min() >= 1 / 255 * (1 - 1e-6)


# ---------------------------------------------------- hand-worked occlusion
def _axis_pair(order):
    s = [0.03, 0.05]
    zoff = [0.0, 0.3]          # camera-space depths 0.5 and 0.8
    sig = [0.7, 0.6]
    rgb = [(1.0, 0.2, 0.1), (0.1, 0.3, 0.9)]
    obj = [[0.0, 2.0, 0.0], [0.0, 0.0, 1.5]]
    idx = list(order)
    sh = np.zeros((2, 1, 3))
    for j, i in enumerate(idx):
        sh[j, 0, :] = (np.array(rgb[i]) - 0.5) / Y00
    sc = make_scene([[0, 0, zoff[i]] for i in idx], [[math.log(s[i])] * 3 for i in idx],
                    opacity=[math.log(sig[i] / (1 - sig[i])) for i in idx], sh=sh,
                    obj=[obj[i] for i in idx], K=2)
    return sc, (s, zoff, sig, rgb, obj)


def test_two_gaussian_occlusion_hand_worked():
    f, z0 = 60.0, 0.5
    sc, (s, zoff, sig, rgb, obj) = _axis_pair((0, 1))
    cam = axis_camera(64, 64, f, z0)
    r = O.OracleScene(sc).render(cam, 0)
    z = [z0 + zoff[0], z0 + zoff[1]]
    a = []
    for i in range(2):
        s32 = float(np.float32(s[i]))
        s2sq = (f * s32 / z[i]) ** 2 + float(np.float32(0.3))
        sg = 1 / (1 + math.exp(-float(np.float32(math.log(sig[i] / (1 - sig[i]))))))
        a.append(sg * math.exp(-0.5 * 0.5 / s2sq))
    c = [np.array([float(np.float32((v - 0.5) / Y00)) * Y00 + 0.5 for v in rgb[i]]) for i in range(2)]
    p = [np.exp(np.array(obj[i], np.float32).astype(np.float64)) for i in range(2)]
    p = [q / q.sum() for q in p]
    C = a[0] * c[0] + (1 - a[0]) * a[1] * c[1]
    A = 1 - (1 - a[0]) * (1 - a[1])
    D = a[0] * z[0] + (1 - a[0]) * a[1] * z[1]
    Op = a[0] * p[0] + (1 - a[0]) * a[1] * p[1]
    Ob = Op.copy(); Ob[0] += 1 - Op.sum()
    np.testing.assert_allclose(r["rgb"][31, 31], C, rtol=1e-6)
    np.testing.assert_allclose(r["alpha"][31, 31], A, rtol=1e-6)
    np.testing.assert_allclose(r["depth"][31, 31], D, rtol=1e-6)
    np.testing.assert_allclose(r["obj"][31, 31], Ob, rtol=1e-6)
    # input order does not matter: the depth sort decides
    sc2, _ = _axis_pair((1, 0))
    r2 = O.OracleScene(sc2).render(cam, 0)
    for k in ("rgb", "alpha", "depth", "obj"):
        np.testing.assert_array_equal(r[k], r2[k])


def test_transmittance_stop_hand_worked():
    """alphas 0.99, 0.98, 0.6 along one ray: after two, T = 2e-4; the third
    would take T to 8e-5 < 1e-4, so it is not blended."""
    f, z0 = 60.0, 0.5
    s = 0.05
    zoff = [0.0, 0.1, 0.2]
    s2 = [(f * float(np.float32(s)) / (z0 + zo)) ** 2 + float(np.float32(0.3)) for zo in zoff]
    e = [math.exp(-0.25 / v) for v in s2]
    want = [0.995, 0.98, 0.6]
    rho = [math.log((w / ee) / (1 - w / ee)) if w / ee < 1 else 8.0 for w, ee in zip(want, e)]
    sc = make_scene([[0, 0, zo] for zo in zoff], [[math.log(s)] * 3] * 3, opacity=rho, K=1)
    cam = axis_camera(64, 64, f, z0)
    r = O.OracleScene(sc).render(cam, 0)
    a = [0.99]
    for i in (1, 2):
        sg = 1 / (1 + math.exp(-float(np.float32(rho[i]))))
        a.append(sg * e[i])
    assert a[1] > 0.979 and a[1] < 0.981 and abs(a[2] - 0.6) < 0.01
    T = (1 - a[0]) * (1 - a[1])
    np.testing.assert_allclose(r["alpha"][31, 31], 1 - T, rtol=1e-9)
    D = a[0] * (z0 + zoff[0]) + (1 - a[0]) * a[1] * (z0 + zoff[1])
    np.testing.assert_allclose(r["depth"][31, 31], D, rtol=1e-6)
    assert r["n_contrib"][31, 31] == 2


# ---------------------------------------------- EWA projection, Monte Carlo
def test_ewa_covariance_matches_projected_samples():
    """The projected 2D covariance (minus the 0.3 px dilation) equals the
    covariance of pinhole-projected samples of a small 3D Gaussian, to first
    order; the mean is the projected centre. The quaternion is unnormalised
    on purpose (it is normalised inside)."""
    rng = np.random.default_rng(3)
    mu = np.array([0.06, -0.04, 0.02])
    logs = np.log(np.array([0.004, 0.002, 0.003]))
    q = np.array([0.9, 0.3, -0.2, 0.4]) * 2.7
    sc = make_scene([mu], [logs], [q], K=1)
    wl = S.make_workload("tiny")
    cams = wl.cand
    for i in range(3):
        v = O.OracleScene(sc).project64(cams, i)[0]
        A, B, C = v[2:5]
        Sig2 = np.linalg.inv(np.array([[A, B], [B, C]])) - 0.3 * np.eye(2)
        qq = (q / np.linalg.norm(q)).astype(np.float32).astype(np.float64)
        w, x, y, z = qq / np.linalg.norm(qq)
        Rq = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                       [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                       [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        assert np.allclose(Rq @ Rq.T, np.eye(3), atol=1e-12)
        s32 = np.exp(np.asarray(logs, np.float32).astype(np.float64))
        pts = np.asarray(mu, np.float32).astype(np.float64) + (
            rng.standard_normal((400_000, 3)) * s32) @ Rq.T
        R = cams.R[i].astype(np.float64); t = cams.t[i].astype(np.float64)
        pc = pts @ R.T + t
        uv = np.stack([cams.fx[i] * pc[:, 0] / pc[:, 2] + cams.cx[i],
                       cams.fy[i] * pc[:, 1] / pc[:, 2] + cams.cy[i]], 1)
        emp = np.cov(uv.T)
        np.testing.assert_allclose(Sig2, emp, rtol=0.02, atol=2e-3 * np.abs(emp).max())
        np.testing.assert_allclose(v[0:2], uv.mean(0), atol=0.01)


def test_decision_path_agrees_with_double_path():
    """The single-precision key path (mean2D, conic, radius, rect, depth
    bits) agrees with the double-precision projection it mirrors."""
    wl = S.make_workload("tiny")
    o = O.OracleScene(wl.scene)
    for i in range(wl.cand.n):
        p32 = o.project32(wl.cand, i)
        v = o.project64(wl.cand, i)
        ok = p32["rect"][:, 0] >= 0
        assert ok.sum() > 100
        np.testing.assert_allclose(p32["mean2d"][ok], v[ok, 0:2], atol=2e-3)
        np.testing.assert_allclose(p32["conic"][ok], v[ok, 2:5], rtol=2e-4,
                                   atol=2e-4 * np.abs(v[ok, 2:5]).max())
        z32 = p32["zbits"][ok].view(np.float32).astype(np.float64)
        np.testing.assert_allclose(z32, v[ok, 6], rtol=1e-6)
        # radius = ceil(3 sqrt(lambda_max)), lambda_max of the 2D covariance
        A, B, C = v[ok, 2], v[ok, 3], v[ok, 4]
        det = A * C - B * B
        a, b, c = C / det, -B / det, A / det
        mid = 0.5 * (a + c)
        lam = mid + np.sqrt(np.maximum(0.1, mid * mid - (a * c - b * b)))
        lam_eig = np.linalg.eigvalsh(np.stack([np.stack([a, b], -1), np.stack([b, c], -1)], -2))[:, 1]
        big = (mid * mid - (a * c - b * b)) > 0.11       # the 0.1 floor is inactive
        np.testing.assert_allclose(lam[big], lam_eig[big], rtol=1e-9)
        r64 = 3 * np.sqrt(lam)
        safe = np.abs(r64 - np.round(r64)) > 1e-3
        np.testing.assert_array_equal(p32["radius"][ok][safe], np.ceil(r64[safe]))


# --------------------------------------------- brute force at tiny sizes
def _brute_lists(p32, W, H, tw=16, th=16):
    rect, zb = p32["rect"], p32["zbits"]
    lists = {}
    for py in range(H):
        for px in range(W):
            tx, ty = px // tw, py // th
            ids = [g for g in range(len(zb)) if rect[g, 0] >= 0 and rect[g, 0] <= tx < rect[g, 1]
                   and rect[g, 2] <= ty < rect[g, 3]]
            ids.sort(key=lambda g: (int(zb[g]), g))
            lists[(px, py)] = ids
    return lists


def _power32(p32, g, px, py):
    f32 = np.float32
    dx = f32(p32["mean2d"][g, 0] - f32(f32(px) + f32(0.5)))
    dy = f32(p32["mean2d"][g, 1] - f32(f32(py) + f32(0.5)))
    A, B, Cc = p32["conic"][g]
    return f32(f32(f32(-0.5) * f32(f32(A * f32(dx * dx)) + f32(Cc * f32(dy * dy)))) - f32(B * f32(dx * dy)))


def _skip32(sc):
    sig32 = (1.0 / (1.0 + np.exp(-sc.opacity.astype(np.float64)))).astype(np.float32)
    return np.log((1.0 / 255.0) / sig32.astype(np.float64)).astype(np.float32)


@pytest.mark.parametrize("seed", [0, 1])
def test_tile_lists_brute_force(seed):
    """Every tile's list is exactly the (depth bits, index)-ordered list of
    the Gaussians whose rectangle covers it (the plain binning rule), and the
    needed sub-list holds exactly those that pass the skip test at one of the
    tile's in-image pixels."""
    sc = random_small_scene(seed, n=30, spread=0.12)
    cam = axis_camera(40, 36, 80.0, 0.5)           # 3x3 tiles, ragged right and bottom
    o = O.OracleScene(sc)
    p32 = o.project32(cam, 0)
    off, ids = o.tile_lists(cam, 0)
    noff, nids = o.tile_needed(cam, 0)
    lists = _brute_lists(p32, 40, 36)
    skip = _skip32(sc)
    GX = 3
    need = {}
    for (px, py), cover in lists.items():
        t = (py // 16) * GX + px // 16
        need.setdefault(t, (cover, set()))
        for g in cover:
            pw = _power32(p32, g, px, py)
            if not (pw > 0 or pw < skip[g]):
                need[t][1].add(g)
    dropped = 0
    for t, (cover, passing) in need.items():
        assert list(ids[off[t]:off[t + 1]]) == cover
        assert list(nids[noff[t]:noff[t + 1]]) == [g for g in cover if g in passing]
        dropped += len(cover) - len(passing)
    assert dropped > 0                              # some rectangle entries are not needed


def _needed_brute(p32, skip, W, H, tw, th):
    """(tile, Gaussian) pairs whose splat passes the skip test at one of the
    tile's in-image pixel centres, by evaluating the single-precision power
    at every pixel of every covered tile (numpy, same operation order)."""
    f32 = np.float32
    GX = (W + tw - 1) // tw
    out = set()
    px = np.arange(W, dtype=np.float32) + f32(0.5)
    py = np.arange(H, dtype=np.float32) + f32(0.5)
    for g in np.nonzero(p32["rect"][:, 0] >= 0)[0]:
        x0, x1, y0, y1 = p32["rect"][g]
        mx, my = p32["mean2d"][g]
        A, B, Cc = p32["conic"][g]
        xs, ys = px[x0 * tw:min(x1 * tw, W)], py[y0 * th:min(y1 * th, H)]
        dx = (mx - xs)[None, :].astype(np.float32)
        dy = (my - ys)[:, None].astype(np.float32)
        q = (A * (dx * dx)).astype(f32) + (Cc * (dy * dy)).astype(f32)
        pw = (f32(-0.5) * q).astype(f32) - (B * (dx * dy)).astype(f32)
        ok = ~((pw > 0) | (pw < skip[g]))
        for yy, xx in zip(*np.nonzero(ok)):
            out.add(((y0 * th + yy) // th * GX + (x0 * tw + xx) // tw, int(g)))
    return out


@pytest.mark.parametrize("aniso", [0.25, 2.5])
def test_tile_needed_elongated_splats(aniso):
    """The needed sub-lists against a vectorised per-pixel brute force, with
    elongated splats (log-scale spread 2.5: axis ratios beyond 1000) where
    the cancellation in the power is largest and a rectangle holds many
    tiles its splat never reaches."""
    rng = np.random.default_rng(7)
    n = 400
    means = np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(-0.1, 0.3, n)], 1)
    log_scales = rng.normal(np.log(0.01), aniso, (n, 3))
    q = rng.standard_normal((n, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = rng.normal(0.0, 1.5, n)
    sh = np.zeros((n, 1, 3)); sh[:, 0, :] = 0.8
    obj = rng.normal(0, 1.0, (n, 2))
    sc = make_scene(means, log_scales, q, opacity, sh, obj, 1, 0)
    W, H = 200, 152
    cam = axis_camera(W, H, 180.0, 1.0)
    o = O.OracleScene(sc)
    p32 = o.project32(cam, 0)
    off, ids = o.tile_lists(cam, 0)
    noff, nids = o.tile_needed(cam, 0)
    got = {(t, int(g)) for t in range(len(noff) - 1) for g in nids[noff[t]:noff[t + 1]]}
    assert got == _needed_brute(p32, _skip32(sc), W, H, 16, 16)
    assert 0 < len(nids) < len(ids)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_composite_brute_force(seed):
    """Per-pixel compositing re-derived in numpy (FP32 decisions from the
    key path, FP64 values) equals the oracle's tile-based render."""
    K = 2
    sc = random_small_scene(seed, n=25, K=K, spread=0.1)
    cam = axis_camera(36, 20, 80.0, 0.5)
    o = O.OracleScene(sc)
    p32 = o.project32(cam, 0)
    v = o.project64(cam, 0)
    r = o.render(cam, 0)
    lists = _brute_lists(p32, 36, 20)
    f32 = np.float32
    sig32 = (1.0 / (1.0 + np.exp(-sc.opacity.astype(np.float64)))).astype(np.float32)
    skip = np.log((1.0 / 255.0) / sig32.astype(np.float64)).astype(np.float32)
    clampt = np.log(f32(0.99).astype(np.float64) / sig32.astype(np.float64)).astype(np.float32)
    p = np.exp(sc.obj_logits.astype(np.float64)); p /= p.sum(1, keepdims=True)
    for (px, py), ids in lists.items():
        T32, T = f32(1.0), 1.0
        C = np.zeros(3); D = 0.0; Op = np.zeros(K + 1)
        for g in ids:
            dx = f32(p32["mean2d"][g, 0] - f32(f32(px) + f32(0.5)))
            dy = f32(p32["mean2d"][g, 1] - f32(f32(py) + f32(0.5)))
            A, B, Cc = p32["conic"][g]
            pw = f32(f32(f32(-0.5) * f32(f32(A * f32(dx * dx)) + f32(Cc * f32(dy * dy)))) - f32(B * f32(dx * dy)))
            if pw > 0 or pw < skip[g]:
                continue
            cl = pw >= clampt[g]
            a32 = f32(0.99) if cl else f32(sig32[g] * f32(math.exp(float(pw))))
            tt = f32(T32 * f32(f32(1.0) - a32))
            if tt < f32(1e-4):
                break
            ddx, ddy = v[g, 0] - (px + 0.5), v[g, 1] - (py + 0.5)
            pw64 = -0.5 * (v[g, 2] * ddx * ddx + v[g, 4] * ddy * ddy) - v[g, 3] * ddx * ddy
            a = 0.99 if cl else v[g, 5] * math.exp(pw64)
            w = a * T
            C += w * v[g, 7:10]; D += w * v[g, 6]; Op += w * p[g]
            T *= 1 - a; T32 = tt
        Ob = Op.copy(); Ob[0] += 1 - Op.sum()
        np.testing.assert_allclose(r["rgb"][py, px], C, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(r["depth"][py, px], D, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(r["alpha"][py, px], 1 - T, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(r["obj"][py, px], Ob, rtol=1e-12, atol=1e-14)


# ------------------------------------------ Jacobian blocks vs finite differences
def _perturbed(sc, g, which, j, h):
    sc2 = S.Scene(sc.means.copy(), sc.log_scales.copy(), sc.quats.copy(), sc.opacity.copy(),
                  sc.sh.copy(), sc.obj_logits.copy(), sc.sh_degree, sc.K)
    arr = getattr(sc2, which)
    flat = arr.reshape(arr.shape[0], -1)
    flat[g, j] = np.float32(flat[g, j] + np.float32(h))
    assert float(flat[g, j]) - float(getattr(sc, which).reshape(arr.shape[0], -1)[g, j]) == h
    return sc2


@pytest.mark.parametrize("seed", [0, 3])
def test_jacobian_blocks_match_finite_differences(seed):
    """A^f_g = sum over pixels and channels of J J^T (Eqs. 6, 9) equals the
    same sum with J from central differences of the rendered outputs
    (decisions frozen; perturbations exactly representable in float32)."""
    K, deg = 2, 1
    sc = random_small_scene(seed, n=5, K=K, deg=deg, spread=0.04)
    cam = axis_camera(40, 34, 90.0, 0.45)
    o = O.OracleScene(sc)
    Ar, Ad, Ao = o.view_blocks(cam, 0)
    fz = o.freeze(cam, 0)
    nb = (deg + 1) ** 2
    h = 2.0 ** -18
    geo = [("means", j) for j in range(3)] + [("log_scales", j) for j in range(3)] + \
          [("quats", j) for j in range(4)] + [("opacity", 0)]
    for g in range(sc.n):
        cols = {"rgb": [], "d": [], "o": []}
        def fd(which, j):
            rp = O.OracleScene(_perturbed(sc, g, which, j, h)).render_frozen(fz, cam, 0)
            rm = O.OracleScene(_perturbed(sc, g, which, j, -h)).render_frozen(fz, cam, 0)
            return {k: (rp[k] - rm[k]) / (2 * h) for k in rp}
        for which, j in geo:
            d = fd(which, j)
            cols["rgb"].append(d["rgb"].reshape(-1))
            cols["d"].append(d["depth"].reshape(-1))
            cols["o"].append(d["obj"].reshape(-1))
        for k in range(nb):
            for ch in range(3):
                cols["rgb"].append(fd("sh", k * 3 + ch)["rgb"].reshape(-1))
        for k in range(K + 1):
            cols["o"].append(fd("obj_logits", k)["obj"].reshape(-1))
        for key, A in (("rgb", Ar[g]), ("d", Ad[g]), ("o", Ao[g])):
            J = np.stack(cols[key], 1)
            Afd = J.T @ J
            scale = max(np.abs(A).max(), 1e-30)
            assert np.abs(A - Afd).max() / scale < 2e-6, (g, key)


# ------------------------------------------------------- IG closed forms
def test_ig_closed_form_single_training_view():
    """With T = {t} and the candidate = t, each Gaussian's gain is
    sum_i log((lambda + 2 c mu_i)/(lambda + c mu_i)) over the eigenvalues of
    A_t (block-diagonal log det, Sec. III-B.1), and the normalised score is
    exactly 1 + beta_d + beta_o (Eq. 10 calibrates a training view to 1)."""
    wl = S.make_workload("tiny")
    sc = wl.scene.subset(np.arange(400))
    o = O.OracleScene(sc)
    train = wl.train.subset([1])
    res = o.score(train, train, delta_view=0)
    c = o.confidence()
    Ar, Ad, Ao = o.view_blocks(train, 0)
    lam = o.hyper.lam
    lam32 = float(np.float32(lam))
    tot = np.zeros(3)
    for f, A in enumerate((Ar, Ad, Ao)):
        mu = np.linalg.eigvalsh(A)
        mu = np.maximum(mu, 0.0)
        per = np.log((lam32 + 2 * c[:, None] * mu) / (lam32 + c[:, None] * mu)).sum(1)
        np.testing.assert_allclose(res["delta"][:, f], per, rtol=1e-8, atol=1e-10)
        tot[f] = per.sum()
    np.testing.assert_allclose(res["ig_cand"][0], tot, rtol=1e-10)
    np.testing.assert_allclose(res["ig_train"][0], tot, rtol=1e-10)
    # (the two block sums run in different thread orders, hence not bit-equal)
    assert abs(res["score"][0] - (1.0 + 10.0 + 1.0)) < 1e-11
    assert res["best"] == 0


def test_ig_general_views_against_dense_slogdet():
    """Two training views and two other candidates: each Gaussian's gain is
    log det(H_T + c A_v) - log det(H_T) with H_T = lambda I + c (A_t0 + A_t1)
    (Eqs. 5, 6, 9), here by LAPACK's LU log-determinant of the dense blocks;
    a training view is scored as H_T + c A_t (counted twice); the score is
    sum_f beta_f IG_f(v) / mean_t IG_f(T, t) (Eqs. 10-11)."""
    wl = S.make_workload("tiny")
    sc = wl.scene.subset(np.arange(300))
    o = O.OracleScene(sc)
    train = wl.train.subset([0, 2])
    cand = wl.cand.subset([1, 4])
    c = o.confidence()
    lam32 = float(np.float32(o.hyper.lam))
    At = [o.view_blocks(train, t) for t in range(2)]
    Av = [o.view_blocks(cand, v) for v in range(2)]

    def gains(HT, A):
        out = np.zeros(sc.n)
        for g in range(sc.n):
            s0 = np.linalg.slogdet(HT[g])
            s1 = np.linalg.slogdet(HT[g] + c[g] * A[g])
            assert s0[0] > 0 and s1[0] > 0
            out[g] = s1[1] - s0[1]
        return out

    igc = np.zeros((2, 3)); igt = np.zeros((2, 3))
    for f in range(3):
        l = At[0][f].shape[1]
        HT = lam32 * np.eye(l)[None] + c[:, None, None] * (At[0][f] + At[1][f])
        for v in range(2):
            per = gains(HT, Av[v][f])
            igc[v, f] = per.sum()
            if v == 1:
                res = o.score(train, cand, delta_view=1)
                np.testing.assert_allclose(res["delta"][:, f], per, rtol=1e-8, atol=1e-10)
        for t in range(2):
            igt[t, f] = gains(HT, At[t][f]).sum()
    res = o.score(train, cand)
    np.testing.assert_allclose(res["ig_cand"], igc, rtol=1e-9)
    np.testing.assert_allclose(res["ig_train"], igt, rtol=1e-9)
    beta = np.array([1.0, o.hyper.beta_d, o.hyper.beta_o])
    want = (igc / igt.mean(0) * beta).sum(1)
    np.testing.assert_allclose(res["score"], want, rtol=1e-9)
    assert res["best"] == int(np.argmax(want))


def test_ig_is_sum_of_nonnegative_gains_and_permutation_invariant():
    wl = S.make_workload("tiny")
    sc = wl.scene.subset(np.arange(300))
    cand = wl.cand.subset([0, 3, 5])
    r1 = O.OracleScene(sc).score(wl.train, cand, delta_view=1)
    assert (r1["delta"] >= -1e-12).all()
    assert (r1["ig_cand"] > 0).all()
    np.testing.assert_allclose(r1["delta"].sum(0), r1["ig_cand"][1], rtol=1e-12)
    perm = np.random.default_rng(0).permutation(sc.n)
    r2 = O.OracleScene(sc.subset(perm)).score(wl.train, cand, delta_view=1)
    np.testing.assert_allclose(r2["ig_cand"], r1["ig_cand"], rtol=1e-10)
    np.testing.assert_allclose(r2["delta"], r1["delta"][perm], rtol=1e-9, atol=1e-12)
    assert r1["best"] == r2["best"] == int(np.argmax(r1["score"]))


def test_object_centric_gating_and_empty_target():
    """Eq. 12: Gaussians whose argmax is not the target gain nothing; a target
    that no Gaussian carries leaves every normaliser at zero."""
    wl = S.make_workload("tiny")
    sc = wl.scene.subset(np.arange(300))
    cand = wl.cand.subset([0, 1])
    o = O.OracleScene(sc, target=2)
    res = o.score(wl.train, cand, delta_view=0)
    am = sc.obj_logits.argmax(1)
    assert np.all(res["delta"][am != 2] == 0.0)
    assert res["best"] in (0, 1)
    sc2 = sc.subset(np.arange(sc.n))
    sc2.obj_logits[:, 3] = -5.0              # nobody carries object 3
    r2 = O.OracleScene(sc2, target=3).score(wl.train, cand)
    assert r2["best"] == -1
    assert np.all(r2["ig_cand"] == 0.0)


def test_invariants_on_tiny_workload():
    wl = S.make_workload("tiny")
    o = O.OracleScene(wl.scene)
    for i in range(0, wl.cand.n, 3):
        r = o.render(wl.cand, i)
        assert np.abs(r["obj"].sum(-1) - 1).max() < 1e-12          # Eq. 2
        assert r["obj"].min() > -1e-12
        assert r["alpha"].min() >= 0 and r["alpha"].max() <= 1
        assert r["rgb"].min() >= 0
        m = r["alpha"] > 1e-6
        zd = r["depth"][m] / r["alpha"][m]
        assert zd.min() > 0.2 and zd.max() < 1.2


@pytest.mark.parametrize("crit", [1, 2])
def test_criterion_variants_closed_form_single_training_view(crit):
    """The criterion variants on T = {t}, candidate = t: per Gaussian
    tr(H_T^-1 c A) = sum_i c mu_i / (lambda + c mu_i) (crit 1) and
    tr(c A) = sum_i c mu_i (crit 2) over the eigenvalues of A_t; the
    normalised score is again exactly 1 + beta_d + beta_o."""
    wl = S.make_workload("tiny")
    sc = wl.scene.subset(np.arange(300))
    o = O.OracleScene(sc, hyper=O.Hyper(crit=crit))
    train = wl.train.subset([2])
    res = o.score(train, train, delta_view=0)
    c = o.confidence()
    lam32 = float(np.float32(o.hyper.lam))
    for f, A in enumerate(o.view_blocks(train, 0)):
        mu = np.maximum(np.linalg.eigvalsh(A), 0.0)
        cm = c[:, None] * mu
        per = (cm / (lam32 + cm)).sum(1) if crit == 1 else cm.sum(1)
        np.testing.assert_allclose(res["delta"][:, f], per, rtol=1e-8, atol=1e-10)
    assert abs(res["score"][0] - 12.0) < 1e-10
