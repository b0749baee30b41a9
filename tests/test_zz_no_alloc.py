"""The tile-key sort that allocates no device memory (nbv_sort_tile_keys_noalloc).

It exists for callers that may not allocate device memory while they run
(applications that reserve the GPU up front under their own allocator, or
latency-critical code where a cudaMalloc, which can synchronise the device,
is not allowed). Its output must equal the tile lists the context's own
sort produces (nbv_debug_tile_lists), bit for bit, on two calls in a row
that share the library's fixed working array. This file is collected last
on purpose.
"""
import numpy as np
import pytest

import nbv_synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2602_08266_gb300 as P
    P.build()
    P.load_library()
    assert torch.cuda.is_available()
    return P


def _keys_from_lists(off, ids, zbits, W, H):
    """The (tile << 32 | depth bits, Gaussian) pairs of the context's tile
    lists, laid out as duplication emits them: Gaussian-index order, each
    Gaussian's tiles in row order."""
    GX = (W + 15) // 16
    ntiles = GX * ((H + 15) // 16)
    tile = np.repeat(np.arange(ntiles, dtype=np.int64), np.diff(off))
    g = ids.astype(np.int64)
    perm = np.lexsort((tile, g))
    tile, g = tile[perm], g[perm]
    keys = (tile.astype(np.uint64) << np.uint64(32)) | zbits[g].astype(np.uint64)
    bits = 1
    while (1 << bits) < ntiles:
        bits += 1
    return keys, g.astype(np.int32), 32 + bits


def _case(P, wl, v):
    sc = P.NBVScorer(wl.scene.K, wl.scene.sh_degree)
    sc.load_scene(wl.scene)
    sc.set_train_views(wl.train)
    sc.set_candidates(wl.cand)
    pr = sc.debug_project(0, v)
    zb = pr["zbits"].cpu().numpy().view(np.uint32)
    off, ids = sc.debug_tile_lists(0, v)
    W, H = int(wl.cand.width[v]), int(wl.cand.height[v])
    ids = ids.cpu().numpy()
    k, val, bits = _keys_from_lists(off.cpu().numpy(), ids, zb, W, H)
    return sc, k, val, bits, ids


@pytest.mark.parametrize("name,scale,v", [("tiny", None, 2), ("scene", 0.02, 5)])
def test_noalloc_sort_matches_context_tile_lists_twice(P, name, scale, v):
    wl = S.make_workload(name, n_views=8, scale=scale)
    sc, k, val, bits, want_ids = _case(P, wl, v)
    assert 0 < len(k) <= P.NOALLOC_MAX_PAIRS
    kin = torch.from_numpy(k.view(np.int64)).cuda()
    vin = torch.from_numpy(val).cuda()
    kin0, vin0 = kin.clone(), vin.clone()
    want_keys = np.sort(k, kind="stable")
    for _ in range(2):                       # two calls in a row share the fixed array
        kout = torch.full_like(kin, -1)
        vout = torch.full_like(vin, -1)
        P.sort_tile_keys_noalloc(kin, vin, bits, kout, vout)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(vout.cpu().numpy(), want_ids)
        np.testing.assert_array_equal(kout.cpu().numpy().view(np.uint64), want_keys)
        assert torch.equal(kin, kin0) and torch.equal(vin, vin0)   # inputs only read
    sc.close()


@pytest.mark.parametrize("n,key_bits", [(1 << 20, 64), (100_003, 24)])
def test_noalloc_sort_largest_input_and_odd_pass_count(P, n, key_bits):
    """The largest input (NBV_NOALLOC_MAX_PAIRS random 64-bit keys with many
    duplicates: eight radix passes, the most histogram and scan scratch) and
    an odd pass count (24 key bits: three passes, the last landing in the
    caller's output) against numpy's stable argsort, twice in a row."""
    assert n <= P.NOALLOC_MAX_PAIRS
    rng = np.random.default_rng(n + key_bits)
    pool = rng.integers(0, 2 ** 63, 4096, dtype=np.int64).view(np.uint64) * np.uint64(2) + np.uint64(1)
    k = pool[rng.integers(0, pool.size, n)]
    mask = np.uint64((1 << key_bits) - 1) if key_bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(k & mask, kind="stable")
    kin = torch.from_numpy(k.view(np.int64)).cuda()
    vin = torch.arange(n, dtype=torch.int32, device="cuda")
    for _ in range(2):
        kout = torch.full_like(kin, -1)
        vout = torch.full_like(vin, -1)
        P.sort_tile_keys_noalloc(kin, vin, key_bits, kout, vout)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(vout.cpu().numpy(), order.astype(np.int32))
        np.testing.assert_array_equal(kout.cpu().numpy().view(np.uint64), k[order])


def test_noalloc_sort_binding_checks(P):
    """Short, strided, wrongly typed or host tensors are refused before the
    library is called."""
    k = torch.zeros(8, dtype=torch.int64, device="cuda")
    v = torch.zeros(8, dtype=torch.int32, device="cuda")
    bad_outputs = [(torch.zeros(4, dtype=torch.int64, device="cuda"), torch.zeros_like(v)),
                   (torch.zeros(16, dtype=torch.int64, device="cuda")[::2], torch.zeros_like(v)),
                   (torch.zeros_like(k), torch.zeros(8, dtype=torch.int64, device="cuda")),
                   (torch.zeros(8, dtype=torch.int64), torch.zeros_like(v))]
    for ko, vo in bad_outputs:
        with pytest.raises(P.NBVError) as e:
            P.sort_tile_keys_noalloc(k, v, 40, ko, vo)
        assert e.value.code == -1


def test_noalloc_sort_rejects_oversized_and_aliased(P):
    lib = P.load_library()
    import ctypes
    k = torch.zeros(8, dtype=torch.int64, device="cuda")
    v = torch.zeros(8, dtype=torch.int32, device="cuda")
    ko = torch.zeros_like(k)
    vo = torch.zeros_like(v)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.nbv_sort_tile_keys_noalloc(p(k), p(v), P.NOALLOC_MAX_PAIRS + 1, 40, p(ko), p(vo), st) == -1
    assert lib.nbv_sort_tile_keys_noalloc(p(k), p(v), 8, 0, p(ko), p(vo), st) == -1
    assert lib.nbv_sort_tile_keys_noalloc(p(k), p(v), 8, 40, p(k), p(vo), st) == -1
    # partial overlaps: an output starting inside an input, or inside the other output
    big = torch.zeros(64, dtype=torch.int64, device="cuda")
    vbig = big.view(torch.int32)
    at = lambda t, i: ctypes.c_void_p(t.data_ptr() + 8 * i)
    assert lib.nbv_sort_tile_keys_noalloc(at(big, 0), p(v), 8, 40, at(big, 4), p(vo), st) == -1
    assert lib.nbv_sort_tile_keys_noalloc(p(k), at(big, 0), 8, 40, at(big, 1), p(vo), st) == -1
    assert lib.nbv_sort_tile_keys_noalloc(p(k), p(v), 8, 40, at(big, 0), at(big, 6), st) == -1
    assert lib.nbv_sort_tile_keys_noalloc(p(k), p(v), 8, 40, at(big, 0), at(big, 8), st) == 0
    torch.cuda.synchronize()
    del vbig
    assert lib.nbv_sort_tile_keys_noalloc(p(k), p(v), 0, 40, p(ko), p(vo), st) == 0
