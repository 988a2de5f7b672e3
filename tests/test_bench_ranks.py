"""Host logic of bench.py's multi-GPU path on the CPU: two ranks over the
gloo backend (the GPU runs use NCCL with one rank per GPU).  Each rank runs
its own batch (weak scaling); the whole-job rate is the units of all ranks
over the slowest rank's time, and only rank 0 runs the reference arm."""
import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 10.0 * (rank + 1)                    # rank 1 is the slow one
        ms = bench.max_over_ranks(my_ms, world, "cpu")
        value = bench.whole_job_value(1000.0, 4, world, ms)
        dist.barrier()
        q.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in res:
        assert ms == 20.0                            # the slowest rank's time
        assert value == pytest.approx(1000.0 * 4 * world / 0.020)


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_value(10.0, 3, 1, 1000.0) == pytest.approx(30.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun every rank but 0 exits without work or output."""
    monkeypatch.setenv("RANK", "1")

    class A:
        warmup, steps, gpus, prec, instances, steps_per_call = 1, 1, 2, "c64", 4096, 256

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(A()) is None
    assert buf.getvalue() == ""
