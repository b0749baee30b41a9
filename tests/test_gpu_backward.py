"""The hand-written backward of the object-aware rasterizer (through the C
ABI): gradients of a loss over colour, depth, opacity and object channels
with respect to every raw parameter, against central finite differences of
the CPU oracle's renders with the forward decisions frozen; the PyTorch
autograd wrapper; and a short map refinement that lowers its loss."""
import numpy as np
import pytest

import nbv_synth as S
from helpers import axis_camera, random_small_scene
from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_08266_gb300 as P
    P.build()
    P.load_library()
    assert torch.cuda.is_available()
    return P


def _perturbed(sc, g, which, j, h):
    sc2 = S.Scene(sc.means.copy(), sc.log_scales.copy(), sc.quats.copy(), sc.opacity.copy(),
                  sc.sh.copy(), sc.obj_logits.copy(), sc.sh_degree, sc.K)
    arr = getattr(sc2, which)
    flat = arr.reshape(arr.shape[0], -1)
    flat[g, j] = np.float32(flat[g, j] + np.float32(h))
    return sc2


@pytest.mark.parametrize("seed", [1, 4])
def test_backward_matches_finite_differences(P, seed):
    K, deg = 2, 1
    sc = random_small_scene(seed, n=10, K=K, deg=deg, spread=0.04)
    cam = axis_camera(40, 34, 90.0, 0.45)
    H, W = 34, 40
    rng = np.random.default_rng(seed + 10)
    wts = dict(rgb=rng.normal(0, 1, (H, W, 3)), depth=rng.normal(0, 1, (H, W)), alpha=rng.normal(0, 1, (H, W)),
               obj=rng.normal(0, 1, (H, W, K + 1)))
    s = P.NBVScorer(K, deg)
    s.load_scene(sc)
    t = {k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in wts.items()}
    g = s.render_backward(cam, 0, t["rgb"], t["depth"], t["alpha"], t["obj"])
    g = {k: v.cpu().numpy().astype(np.float64).reshape(sc.n, -1) for k, v in g.items()}
    o = O.OracleScene(sc)
    fz = o.freeze(cam, 0)

    def loss(scene):
        r = O.OracleScene(scene).render_frozen(fz, cam, 0)
        return sum(float((r[k] * wts[k]).sum()) for k in wts)

    h = 2.0 ** -14
    for which in ("means", "log_scales", "quats", "opacity", "sh", "obj_logits"):
        cols = g[which].shape[1]
        fd = np.zeros((sc.n, cols))
        for gi in range(sc.n):
            for j in range(cols):
                fd[gi, j] = (loss(_perturbed(sc, gi, which, j, h)) - loss(_perturbed(sc, gi, which, j, -h))) / (2 * h)
        scale = np.abs(fd).max() + 1e-12
        err = np.abs(g[which] - fd).max() / scale
        assert err < 2e-3, (which, err)
    s.close()


def test_autograd_function_and_refinement(P):
    """torch.autograd through the library's backward equals the direct call;
    Adam on L1 colour + L1 depth + object cross-entropy against renders of a
    perturbed copy of the scene lowers the loss."""
    from paper_2602_08266_gb300 import diff
    wl = S.make_workload("tiny")
    sc = wl.scene
    rng = np.random.default_rng(0)
    truth = S.Scene(sc.means + rng.normal(0, 0.005, sc.means.shape).astype(np.float32), sc.log_scales.copy(),
                    sc.quats.copy(), (sc.opacity + rng.normal(0, 0.1, sc.opacity.shape)).astype(np.float32),
                    sc.sh.copy(), sc.obj_logits.copy(), sc.sh_degree, sc.K)
    s = P.NBVScorer(sc.K, sc.sh_degree)
    s.load_scene(truth)
    cams = wl.train
    tgt = [s.render_camera(cams, i) for i in range(cams.n)]
    ids = [t["obj"].argmax(-1) for t in tgt]
    params = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().requires_grad_(True)
              for a in (sc.means, sc.log_scales, sc.quats, sc.opacity, sc.sh, sc.obj_logits)]

    def total_loss():
        L = 0.0
        for i in range(cams.n):
            rgb, depth, alpha, obj = diff.render(s, cams, i, *params)
            ce = -(torch.log(obj.clamp_min(1e-6)).gather(-1, ids[i][..., None])).mean()
            L = L + (rgb - tgt[i]["rgb"]).abs().mean() + (depth - tgt[i]["depth"]).abs().mean() + 0.1 * ce
        return L

    # autograd equals the direct backward for one view
    rgb, depth, alpha, obj = diff.render(s, cams, 0, *params)
    (rgb.sum() + 2 * depth.sum() + 3 * obj[..., 1].sum()).backward()
    s.load_scene(sc)
    gr = torch.ones_like(rgb)
    gd = torch.full_like(depth, 2.0)
    go = torch.zeros_like(obj)
    go[..., 1] = 3.0
    g = s.render_backward(cams, 0, gr, gd, None, go)
    # Both calls add the same per-tile terms with float atomics, in an order
    # that differs from run to run: where the terms cancel, the difference
    # scales with their magnitudes rather than with the sum, so the absolute
    # tolerance follows the tensor's largest entry.
    for p, k in zip(params, ("means", "log_scales", "quats", "opacity", "sh", "obj_logits")):
        ref = g[k].reshape(-1)
        torch.testing.assert_close(p.grad.reshape(-1), ref, rtol=1e-5,
                                   atol=1e-6 + 1e-5 * float(ref.abs().max()))
        p.grad = None
    opt = torch.optim.Adam(params, lr=2e-3)
    with torch.no_grad():
        l0 = float(total_loss())
    for _ in range(30):
        opt.zero_grad()
        L = total_loss()
        L.backward()
        opt.step()
    with torch.no_grad():
        l1 = float(total_loss())
    assert l1 < 0.8 * l0, (l0, l1)
    s.close()


def test_backward_on_a_1000_gaussian_crop_of_the_500k_scene(P):
    """The backward on the 500,000-Gaussian table-top scene's densest
    region: the 1,000 Gaussians nearest the first observed view's central
    ray, rendered at 640x480 with K=32 objects and SH degree 3. Per
    parameter type, 16 sampled (Gaussian, component) pairs among the
    Gaussians with the larger gradients, and 4 random directions over all
    1,000 Gaussians, against FP64 central differences of the oracle's frozen
    renders. The perturbation actually applied is the float32 difference,
    so rounding of the perturbed parameters does not enter the comparison."""
    wl = S.make_workload("diff", seed=0)
    full, cams = wl.scene, wl.train
    pc = full.means @ cams.R[0].T + cams.t[0]
    ray = np.where(pc[:, 2] > 0.1, np.hypot(pc[:, 0] / pc[:, 2], pc[:, 1] / pc[:, 2]), np.inf)
    c = int(np.argmin(ray))
    sc = full.subset(np.sort(np.argsort(np.linalg.norm(full.means - full.means[c], axis=1))[:1000]))
    H, W = int(cams.height[0]), int(cams.width[0])
    rng = np.random.default_rng(42)
    wts = dict(rgb=rng.normal(0, 1, (H, W, 3)), depth=rng.normal(0, 1, (H, W)), alpha=rng.normal(0, 1, (H, W)),
               obj=rng.normal(0, 1, (H, W, sc.K + 1)))
    s = P.NBVScorer(sc.K, sc.sh_degree)
    s.load_scene(sc)
    t = {k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in wts.items()}
    g = s.render_backward(cams, 0, t["rgb"], t["depth"], t["alpha"], t["obj"])
    g = {k: v.cpu().numpy().astype(np.float64).reshape(sc.n, -1) for k, v in g.items()}
    s.close()
    fz = O.OracleScene(sc).freeze(cams, 0)

    def loss(scene):
        r = O.OracleScene(scene).render_frozen(fz, cams, 0)
        return sum(float((r[k] * wts[k]).sum()) for k in wts)

    def shifted(which, delta):
        """The scene with `delta` added to one parameter array in float32,
        and the perturbation that float32 actually applied."""
        sc2 = S.Scene(sc.means.copy(), sc.log_scales.copy(), sc.quats.copy(), sc.opacity.copy(),
                      sc.sh.copy(), sc.obj_logits.copy(), sc.sh_degree, sc.K)
        arr = getattr(sc2, which)
        base = arr.reshape(sc.n, -1).astype(np.float64)
        new = (base + delta).astype(np.float32)
        arr.reshape(sc.n, -1)[...] = new
        return sc2, new.astype(np.float64) - base

    h = 2.0 ** -14
    for which in ("means", "log_scales", "quats", "opacity", "sh", "obj_logits"):
        gw = g[which]
        cols = gw.shape[1]
        row = np.abs(gw).max(1)
        strong = np.nonzero(row >= np.quantile(row, 0.75))[0]
        assert row.max() > 0, which
        scale = np.abs(gw).max()
        for _ in range(16):
            gi, j = int(rng.choice(strong)), int(rng.integers(cols))
            e = np.zeros((sc.n, cols))
            e[gi, j] = h
            sp, dp = shifted(which, e)
            sm, dm = shifted(which, -e)
            fd = (loss(sp) - loss(sm)) / (dp[gi, j] - dm[gi, j])
            assert abs(gw[gi, j] - fd) <= 2e-3 * scale, (which, gi, j, gw[gi, j], fd, scale)
        for _ in range(4):
            v = rng.normal(0, 1, (sc.n, cols))
            sp, dp = shifted(which, h * v)
            sm, dm = shifted(which, -h * v)
            fd = loss(sp) - loss(sm)
            lin = float((gw * (dp - dm)).sum())
            # errors in single entries add up like a random walk over the
            # terms, so the bar follows the terms' 2-norm
            mag = float(np.linalg.norm(gw * (dp - dm)))
            assert abs(lin - fd) <= 1e-3 * abs(fd) + 1e-2 * mag, (which, lin, fd, mag)
