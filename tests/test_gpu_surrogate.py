"""The learned candidate pre-scoring on the GPU, through the C ABI: the
tcgen05 BF16 GEMM against a CPU product, the descriptors and the MLP's
forward pass and gradients against the CPU oracle, training, and what the
trained network gains over scoring every candidate exactly."""
import numpy as np
import pytest

import nbv_synth as S
from oracle import oracle as O
from oracle import surrogate as SO

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_08266_gb300 as P
    P.build()
    P.load_library()
    assert torch.cuda.is_available()
    return P


def _bf(a):
    return torch.from_numpy(SO.bf16(a.astype(np.float32))).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M,N,K,ta,tb", [(128, 256, 64, False, False), (200, 160, 100, False, False),
                                          (256, 320, 512, True, False), (77, 48, 300, True, True),
                                          (130, 16, 16, False, True)])
def test_gemm_bf16_tcgen05(P, M, N, K, ta, tb):
    rng = np.random.default_rng(M * 7 + N + K)
    a = SO.bf16(rng.normal(0, 1, (M, K)).astype(np.float32))
    b = SO.bf16(rng.normal(0, 1, (N, K)).astype(np.float32))
    A = _bf(a.T.copy() if ta else a)
    B = _bf(b.T.copy() if tb else b)
    a_str = (1, M) if ta else (K, 1)
    b_str = (1, N) if tb else (K, 1)
    D = P.gemm_bf16(A, a_str, B, b_str, M, N, K).cpu().numpy().astype(np.float64)
    want = a.astype(np.float64) @ b.astype(np.float64).T
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T
    assert np.all(np.abs(D - want) <= 1e-4 * scale + 1e-6)


def test_gemm_bounded_wait_runs_out_and_device_stays_usable(P):
    """The first wait for the tensor cores' commit given no polls gives up
    at once: the launch records the time-out (NBV_ERR_TIMEOUT), drains what
    it has in flight with the full bound and frees its tensor memory; with
    the default restored the same product is exact again, and an MLP forward
    pass still works."""
    rng = np.random.default_rng(3)
    a = SO.bf16(rng.normal(0, 1, (200, 96)).astype(np.float32))
    b = SO.bf16(rng.normal(0, 1, (48, 96)).astype(np.float32))
    A, B = _bf(a), _bf(b)
    try:
        P.set_gemm_wait_polls(0)
        for _ in range(2):
            with pytest.raises(P.NBVError) as e:
                P.gemm_bf16(A, (96, 1), B, (96, 1), 200, 48, 96)
            assert e.value.code == -5
    finally:
        P.set_gemm_wait_polls(-1)
    D = P.gemm_bf16(A, (96, 1), B, (96, 1), 200, 48, 96).cpu().numpy().astype(np.float64)
    want = a.astype(np.float64) @ b.astype(np.float64).T
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T
    assert np.all(np.abs(D - want) <= 1e-4 * scale + 1e-6)
    mlp = P.MLP(96, 64, seed=1)
    y = mlp.forward(torch.from_numpy(a).cuda())
    assert torch.isfinite(y).all()
    mlp.close()


@pytest.mark.parametrize("name,target,scale", [("tiny", -1, None), ("tiny", 2, None), ("scene", -1, 0.05)])
def test_descriptors_match_oracle(P, name, target, scale):
    wl = S.make_workload(name, n_views=12, scale=scale)
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    sc.prepare(target)
    d = sc.descriptors().cpu().numpy().astype(np.float64)
    o = O.OracleScene(wl.scene, target=target)
    obs = sum(o.view_w2(wl.train, t) for t in range(wl.train.n))
    want = SO.descriptors(wl.scene, wl.cand, o.confidence(), obs, wl.train)
    exact = np.r_[0:192, 384:440]          # cells and object bins: same decisions, sums in another order
    np.testing.assert_allclose(d[:, exact], want[:, exact], rtol=2e-5, atol=1e-6)
    # the training-coverage blocks: the kernel's w^2 sums come from its TF32
    # contraction; the novelty (1 - cos) from single-precision directions
    np.testing.assert_allclose(d[:, 192:384], want[:, 192:384], rtol=2e-3, atol=2e-4)
    np.testing.assert_allclose(d[:, 440:], want[:, 440:], rtol=2e-3, atol=2e-4)
    sc.close()


def test_mlp_forward_and_gradients_match_oracle(P):
    rng = np.random.default_rng(5)
    mlp = P.MLP(320, 256, seed=11)
    p = mlp.get_params().cpu().numpy().astype(np.float64)
    B = 300
    x = rng.normal(0, 1, (B, 320)).astype(np.float32)
    t = rng.normal(0, 1, B).astype(np.float32)
    y = mlp.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    yo, _ = SO.forward(p, x, 320, 256)
    np.testing.assert_allclose(y, yo, rtol=0, atol=2e-2 * (np.abs(yo).max() + 1e-3))
    g, loss = mlp.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    go, lo = SO.gradients(p, x, t, 320, 256)
    assert loss == pytest.approx(lo, rel=2e-2)
    o = SO.layout(320, 256)
    for a, b in (("W1", "b1"), ("b1", "W2"), ("W2", "b2"), ("b2", "w3"), ("w3", "b3"), ("b3", "P")):
        gs, ws = g[o[a]:o[b]], go[o[a]:o[b]]
        err = np.linalg.norm(gs - ws) / (np.linalg.norm(ws) + 1e-12)
        assert err < 2e-2, (a, err)
    mlp.close()


def test_mlp_training_reduces_loss(P):
    rng = np.random.default_rng(6)
    mlp = P.MLP(320, 256, seed=1)
    x = torch.from_numpy(rng.normal(0, 1, (2048, 320)).astype(np.float32)).cuda()
    w = torch.from_numpy(rng.normal(0, 1, 320).astype(np.float32)).cuda()
    t = torch.tanh(x @ w / 8.0).contiguous()
    from paper_2602_08266_gb300 import surrogate as SG
    losses = SG.train(mlp, x, t, steps=300, batch=256, lr=1e-3)
    assert losses[-1] < 0.1 * losses[0], losses
    mlp.close()


def test_pruned_scoring_gain(P):
    """Trained on exact scores of 32 seeded small scenes (128 candidates
    each), the network keeps 16 of 128 candidates of unseen scenes; the
    exact best candidate must be among them far more often than for a
    random choice of 16 (12.5%), and nbv_score_pruned must return it."""
    from paper_2602_08266_gb300 import surrogate as SG
    xs, zs = [], []
    for s in range(32):
        wl = S.make_workload("tiny", seed=100 + s, n_views=128)
        x, z, _ = SG.scene_labels(P, wl)
        xs.append(x)
        zs.append(z)
    X, Y = torch.cat(xs), SG.rank_target(torch.cat(zs))
    mlp = P.MLP(448, 256, seed=3)
    losses = SG.train(mlp, X, Y, steps=600, batch=512, lr=1e-3)
    assert losses[-1] < 0.8 * losses[0]
    hit = agree = 0
    trials = 12
    for s in range(trials):
        wl = S.make_workload("tiny", seed=900 + s, n_views=128)
        _, _, y = SG.scene_labels(P, wl)
        best_exact = int(torch.argmax(y).item())
        sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree, batched=1)
        sc.load_scene(wl.scene)
        sc.set_train_views(wl.train)
        sc.set_candidates(wl.cand)
        sc.prepare(-1)
        r = sc.score_pruned(mlp, 16)
        sc.close()
        hit += int(best_exact in set(r["kept"].tolist()))
        agree += int(r["best"] == best_exact)
    print(f"exact best kept in {hit}/{trials}, pruned argmax agrees in {agree}/{trials}")
    assert agree >= hit - 1
    assert hit >= 0.5 * trials
    mlp.close()
