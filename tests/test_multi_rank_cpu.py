"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1) run
the per-rank mock choice, the max-over-ranks step time and the whole-job
per-mock value exactly as the GPU ranks do (there only the device of the
reduced tensor differs)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        step_ms = [120.0, 150.0][rank]
        t = bench.max_over_ranks(step_ms, dist, torch, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.mock_seed(7, rank))
        out.put((rank, t, bench.per_mock(t, world), seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, seeds in res:
        assert t == 150.0          # the slowest rank sets the step time
        assert v == 75.0           # two mocks per step
        assert seeds == [7, 8]     # one mock per rank


def test_single_process_has_no_reduction():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, torch, "cpu") == 3.5
    assert bench.per_mock(10.0, 1) == 10.0
