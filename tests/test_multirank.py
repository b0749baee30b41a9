"""The multi-rank harness of bench.py on CPU ranks (gloo, world size 2):
candidate sets differ per rank and are reproducible, the step time taken is
the maximum over ranks, the whole-job throughput counts every rank's views,
and the reference arm does its work on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import bench
    import nbv_synth as S
    wl = S.make_workload("tiny")
    cand = bench.rank_candidates(S, np, wl, rank, world)
    again = bench.rank_candidates(S, np, wl, rank, world)
    t = bench.max_over_ranks(torch, 10.0 + 5.0 * rank, world, torch.device("cpu"))
    gathered = [None] * world
    dist.all_gather_object(gathered, np.asarray(cand.t).tolist())
    out[rank] = dict(t=t, same_again=bool(np.array_equal(cand.t, again.t)), n=int(cand.n),
                     distinct=gathered[0] != gathered[1], world_seen=bench.dist_info()[0])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        assert res[r]["t"] == 15.0                 # the slowest rank's time on every rank
        assert res[r]["same_again"] and res[r]["n"] == 8
        assert res[r]["distinct"]                  # each rank scores its own candidates
        assert res[r]["world_seen"] == world


def test_job_throughput_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(64, 4, 5, 1000.0) == pytest.approx(64 * 4 * 5)


def test_reference_arm_is_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


def test_roofline_work_counts():
    """The roofline's algorithmic counts: 16 + (K+1) flops per forward pair
    and 110 + 8 (K+1) per information pair on the FP32 pipes (the scope
    table's constants), 2 (88 + 6 K) tensor flops per information pair, the
    projection's bytes (parameters once, 44 B per (view, Gaussian)) and a
    plain binning sort's bytes (ceil(bits / 8) passes of 2 x 12 B)."""
    sys.path.insert(0, ROOT)
    import bench
    st = {"pairs_evaluated": 1000, "pairs_information": 10}
    assert bench.composite_fp32_flops(st, 16) == 1000 * 33 + 10 * 246
    assert bench.composite_fp32_flops({"pairs_evaluated": 0, "pairs_information": 0}, 16) == 0
    assert bench.composite_tensor_flops(st, 32) == 10 * 2 * 280
    assert bench.project_bytes(10, 4, 3) == 10 * 240 + 44 * 40
    # 256 views (8 bits) and 192,000 tiles (18 bits) + 32 depth bits: 58 bits, 8 passes
    assert bench.sort_bytes(100, 256, 192_000) == 8 * 24 * 100
