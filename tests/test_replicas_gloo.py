"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
solves its own replica of the workload (the grids of CTMGRIT^loc are
independent, Alg. 3), so the only exchange is the max of the step times;
the whole-job value counts the units of all ranks over that max.  The
reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]
        slow = bench.max_over_ranks(ms, world)
        value = bench.job_value(1000.0, world, slow)
        # the reference arm: rank 0 alone does the work and reports
        args = type("A", (), {"workload": 1, "steps": 1, "warmup": 0})()
        ref = bench.run_reference(args, rank, world) if rank == 1 else None
        q.put((rank, slow, value, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, value, ref in out:
        assert slow == 17.25                          # every rank sees the slowest time
        assert value == pytest.approx(2 * 1000.0 / 0.01725)
        assert ref is None                            # non-zero ranks exit without work


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_value(500.0, 1, 2.0) == pytest.approx(250000.0)
